// stencil_kernels.cu - the FP64 stencil steps of the projection (FluTAS Sec. 3.3):
// density coefficients (rho0 = min rho, (1 - rho0/rho_f)/h per face), the split
// right-hand side f = (rho0/dt) D u** + D[(1 - rho0/rho_f) G p_hat] and the correction
// u^{n+1} = u** - (dt/rho0)[G p - (1 - rho0/rho_f) G p_hat].
//
// On GB300 the FP64 pipe (about 0.5 T lane-ops/s) rather than HBM bounds these kernels,
// so they are written to minimise FP64 instructions per cell:
//   * the per-face division of rho0/rho_f is done once per density update (set_density),
//     with an FP32 seed and two FP64 Newton steps, and stored as bx, by, bz;
//   * p~ = (dt/rho0) p_hat is evaluated once per cell into a shared-memory plane;
//   * each face flux q = u + b (p~_+ - p~) is evaluated once and shared by the two cells
//     that it separates (x and y faces through shared memory, z faces carried in a
//     register while the CTA marches up a column of planes).
#include "flups_impl.cuh"

namespace {

// 1/s for s in the normal FP32 range: FP32 hardware seed (rcp.approx) refined by two
// Newton-Raphson steps y <- y + y (1 - s y) in FP64 (each step squares the relative error).
// The FP64 <-> FP32 conversions of the seed are done on the bit patterns with integer
// operations (truncating s to 24 bits and widening y exactly), since GB300's conversion
// instructions run on the narrow FP64 pipe; the seed only needs ~2^-22 relative accuracy.
__device__ __forceinline__ double recip64(double s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    const unsigned int hi = (unsigned int)(b >> 32);
    const unsigned int e = (hi >> 20) & 0x7FFu;                    // 897 <= e <= 1150 (normal FP32)
    const float sf = __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | ((unsigned int)(b >> 29) & 0x7FFFFFu));
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(sf));
    const unsigned int yb = __float_as_uint(yf);
    const unsigned int ye = (yb >> 23) & 0xFFu;
    double y = __hiloint2double((int)((yb & 0x80000000u) | ((ye + 896u) << 20) | ((yb & 0x7FFFFFu) >> 3)),
                                (int)((yb & 7u) << 29));
    double e1 = fma(-s, y, 1.0);
    y = fma(y, e1, y);
    e1 = fma(-s, y, 1.0);
    return fma(y, e1, y);
}

// Fixed point for exact stencil sums at a per-cell scale: x * 2^(1080 - emax) truncated toward
// zero as a 64-bit integer, for a binary64 x whose biased exponent is at most emax (so
// |result| < 2^58 and sums of up to 32 such values cannot overflow).  Integer operations only.
__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }
__device__ __forceinline__ long long fixe(double x, int emax) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (e ? 0x10000000000000LL : 0LL);
    const int d = emax - (e ? e : 1);
    const long long X = d >= 64 ? 0LL : ((m << 5) >> d);
    return b < 0 ? -X : X;
}

// Valid densities: finite and within [1e-30, 1e30] (so the FP32 seed above is normal).
// Positive doubles order like their bit patterns, so the test is two integer compares.
__device__ __forceinline__ bool rho_bad(double r) {
    const long long b = __double_as_longlong(r);
    return b < 0x39B4484BFEEBC2A0LL || b > 0x46293E5939A08CEALL;   // 1e-30, 1e30
}

// One CTA per stencil tile (RX x TY cells of a plane, KC planes): the tile's density range
// over the cells whose values its rhs and correct CTAs read (the tile and its one-cell halo
// in -x, +x, -y, +y, -z, +z, no edges or corners), as binary64 bit patterns (positive
// doubles order like their bit patterns, so min and max are integer compares); and, over
// the tile's own cells only, the partial minimum and the invalid-density flag for rho0.
// A tile whose range is [rho0, rho0] has every face coefficient (1 - rho0/rho_f) equal to
// zero.  trange[2t] = min, trange[2t+1] = max; part[2t] = min over own cells, part[2t+1] = bad.
template <int RX>
__global__ void __launch_bounds__(RX * FLUPS_TY) k_rho_tiles(const double* __restrict__ rho, Geo g,
                                                             long long* __restrict__ trange,
                                                             long long* __restrict__ part) {
    constexpr int TY = FLUPS_TY, KC = FLUPS_KC;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * RX, j0 = blockIdx.y * TY;
    const int kb = blockIdx.z * KC, ke = min(kb + KC, g.nz);
    const int nx = g.nx, ny = g.ny;
    const int i = i0 + tx, j = j0 + ty;
    const long long BIG = 0x7FFFFFFFFFFFFFFFLL;
    long long mn_own = BIG, mn = BIG, mx = -BIG;
    int bad = 0;
    // x and y halo cells of this thread (lanes at the tile's x edges, rows at its y edges)
    const int ih = tx == 0 ? wrapm(i0 - 1, nx) : (tx == RX - 1 ? wrapm(i0 + RX, nx) : -1);
    const int jh = ty == 0 ? wrapm(j0 - 1, ny) : (ty == TY - 1 ? wrapm(j0 + TY, ny) : -1);
    for (int k = kb; k < ke; ++k) {
        const size_t pl = (size_t)k * ny;
        const double r = __ldg(rho + (pl + j) * nx + i);
        const long long b = __double_as_longlong(r);
        mn_own = b < mn_own ? b : mn_own;
        bad |= rho_bad(r);
        mx = b > mx ? b : mx;
        if (ih >= 0) {
            const long long h = __double_as_longlong(__ldg(rho + (pl + j) * nx + ih));
            mn = h < mn ? h : mn;
            mx = h > mx ? h : mx;
        }
        if (jh >= 0) {
            const long long h = __double_as_longlong(__ldg(rho + (pl + jh) * nx + i));
            mn = h < mn ? h : mn;
            mx = h > mx ? h : mx;
        }
    }
    mn = mn_own < mn ? mn_own : mn;
    // z halo planes (a wall has no plane beyond it)
    const bool lo = !(g.walls && kb == 0), hi = !(g.walls && ke == g.nz);
    if (lo) {
        const int k = kb == 0 ? g.nz - 1 : kb - 1;
        const long long h = __double_as_longlong(__ldg(rho + ((size_t)k * ny + j) * nx + i));
        mn = h < mn ? h : mn;
        mx = h > mx ? h : mx;
    }
    if (hi) {
        const int k = ke == g.nz ? 0 : ke;
        const long long h = __double_as_longlong(__ldg(rho + ((size_t)k * ny + j) * nx + i));
        mn = h < mn ? h : mn;
        mx = h > mx ? h : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long t = __shfl_xor_sync(0xffffffffu, mn_own, o);
        mn_own = t < mn_own ? t : mn_own;
        t = __shfl_xor_sync(0xffffffffu, mn, o);
        mn = t < mn ? t : mn;
        t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    constexpr int NW = RX * TY / 32;
    __shared__ long long s_own[NW], s_mn[NW], s_mx[NW];
    __shared__ int s_bad[NW];
    const int tid = ty * RX + tx, lane = tid & 31, wid = tid >> 5;
    if (lane == 0) { s_own[wid] = mn_own; s_mn[wid] = mn; s_mx[wid] = mx; s_bad[wid] = bad; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < NW; ++w) {
            mn_own = s_own[w] < mn_own ? s_own[w] : mn_own;
            mn = s_mn[w] < mn ? s_mn[w] : mn;
            mx = s_mx[w] > mx ? s_mx[w] : mx;
            bad |= s_bad[w];
        }
        const int t = (blockIdx.z * g.tny + blockIdx.y) * g.tnx + blockIdx.x;
        trange[2 * t] = mn;
        trange[2 * t + 1] = mx;
        part[2 * t] = mn_own;
        part[2 * t + 1] = bad;
    }
}

__global__ void __launch_bounds__(1024) k_rho_finalize(const long long* __restrict__ part, int nblk, DevScalars* sc,
                                                       double rho0_user, double idx, double idy) {
    long long mn = 0x7FFFFFFFFFFFFFFFLL;
    int bad = 0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        mn = part[2 * i] < mn ? part[2 * i] : mn;
        bad |= (int)part[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, mn, o);
        mn = t < mn ? t : mn;
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ long long smn[32];
    __shared__ int sbad[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { smn[wid] = mn; sbad[wid] = bad; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        mn = smn[w] < mn ? smn[w] : mn;
        bad |= sbad[w];
    }
    const double r0 = rho0_user > 0.0 ? rho0_user : __longlong_as_double(mn);
    sc->rho0 = r0;
    sc->inv_rho0 = 1.0 / r0;
    sc->m2r0 = -2.0 * r0;
    sc->m2r0_dx = -2.0 * r0 * idx;
    sc->m2r0_dy = -2.0 * r0 * idy;
    sc->bad_rho = bad;
}

// True when every face coefficient a tile's CTA reads is zero: the tile's density range
// (cells and one-cell halo) is exactly [rho0, rho0].
__device__ __forceinline__ bool tile_uniform(const Geo& g, const DevScalars* __restrict__ sc) {
    const int t = (blockIdx.z * g.tny + blockIdx.y) * g.tnx + blockIdx.x;
    const long long b0 = __double_as_longlong(sc->rho0);
    return g.trange[2 * t] == b0 && g.trange[2 * t + 1] == b0;
}

// The three coefficients of one cell when some face has a density other than rho0.  Kept
// out of line so that the compiler does not evaluate the reciprocals speculatively in the
// (common) warps where every face is at rho0.
__device__ __noinline__ double3 face_coeffs_slow(double rc, double re, double rn, double rt, double iz, bool nx_,
                                                 bool ny_, bool nz_, const DevScalars* __restrict__ sc, double idx,
                                                 double idy) {
    double3 v = make_double3(0.0, 0.0, 0.0);
    if (nx_) v.x = fma(sc->m2r0_dx, recip64(rc + re), idx);
    if (ny_) v.y = fma(sc->m2r0_dy, recip64(rc + rn), idy);
    if (nz_) v.z = iz * fma(sc->m2r0, recip64(rc + rt), 1.0);
    return v;
}

// b = (1 - rho0/rho_f) / h = 1/h - (2 rho0 / h) / (rho_a + rho_b) for the face above each
// cell in x, y and z (b = 0 on the top wall face), written only inside flagged tiles and on
// their one-cell lower halo in x, y and z: exactly the coefficients the rhs and correct
// kernels read.  One CTA per tile, RX x TY threads marching up the tile's planes.
template <int RX>
__global__ void __launch_bounds__(RX * FLUPS_TY) k_face_coeffs(const double* __restrict__ rho,
                                                               double* __restrict__ bx, double* __restrict__ by,
                                                               double* __restrict__ bz, Geo g,
                                                               const DevScalars* __restrict__ sc) {
    if (tile_uniform(g, sc)) return;
    const int i0 = blockIdx.x * RX, j0 = blockIdx.y * FLUPS_TY;
    const int kb = blockIdx.z * FLUPS_KC, ke = min(kb + FLUPS_KC, g.nz);
    const int k_lo = (g.walls && kb == 0) ? 0 : kb - 1;
    const long long b0 = __double_as_longlong(sc->rho0);
    const int tid = threadIdx.y * RX + threadIdx.x, nthr = RX * FLUPS_TY;
    constexpr int W = RX + 1, Hh = FLUPS_TY + 1;
    for (int kk = k_lo; kk < ke; ++kk) {
        const int k = kk < 0 ? g.nz - 1 : kk;
        const int kp = g.walls ? (k + 1 < g.nz ? k + 1 : k) : (k + 1 == g.nz ? 0 : k + 1);
        const double iz = __ldg(g.idzc + k);
        for (int e = tid; e < W * Hh; e += nthr) {
            const int bb = e / W, aa = e - bb * W;
            const int i = wrapm(i0 - 1 + aa, g.nx), j = wrapm(j0 - 1 + bb, g.ny);
            const size_t idx = ((size_t)k * g.ny + j) * g.nx + i;
            const long long bc_ = __double_as_longlong(__ldg(rho + idx));
            const long long be = __double_as_longlong(__ldg(rho + ((size_t)k * g.ny + j) * g.nx + (wrapm(i + 1, g.nx))));
            const long long bn = __double_as_longlong(__ldg(rho + ((size_t)k * g.ny + (wrapm(j + 1, g.ny))) * g.nx + i));
            const long long bt = __double_as_longlong(__ldg(rho + ((size_t)kp * g.ny + j) * g.nx + i));
            const bool cz0 = bc_ == b0;
            const bool need_x = !(cz0 && be == b0), need_y = !(cz0 && bn == b0);
            const bool need_z = !(cz0 && bt == b0) && __double_as_longlong(iz) != 0;
            double3 v = make_double3(0.0, 0.0, 0.0);
            if (__any_sync(__activemask(), need_x || need_y || need_z))
                v = face_coeffs_slow(__longlong_as_double(bc_), __longlong_as_double(be), __longlong_as_double(bn),
                                     __longlong_as_double(bt), iz, need_x, need_y, need_z, sc, g.idx, g.idy);
            bx[idx] = v.x;
            by[idx] = v.y;
            bz[idx] = v.z;
        }
    }
}

// ------------------------------------------------------------------------- rhs
// CTA = RX x TY cells of one plane, marching up KC planes.  Shared memory holds p~ on an
// extended plane (cells j0-1 .. j0+TY, i0-1 .. i0+RX) for the current and the next level,
// and the x- and y-face fluxes of the current level.  A tile with every face coefficient
// zero has q = u on all its faces and reduces to f = (rho0/dt) D u (same bits).
template <int RX, int TY>
__global__ void __launch_bounds__(RX * TY) k_rhs(const double* __restrict__ u, const double* __restrict__ v,
                                                 const double* __restrict__ w, const double* __restrict__ pn,
                                                 const double* __restrict__ pnm1, const double* __restrict__ bx,
                                                 const double* __restrict__ by, const double* __restrict__ bz,
                                                 double* __restrict__ f, Geo g, double c1, double c2, double dt,
                                                 double inv_dt, const DevScalars* __restrict__ sc) {
    __shared__ double Pt[2][TY + 2][RX + 2];
    __shared__ double QX[TY][RX + 1];
    __shared__ double QY[TY + 1][RX];
    constexpr int KC = FLUPS_KC;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RX + tx, nthr = RX * TY;
    const int i0 = blockIdx.x * RX, j0 = blockIdx.y * TY;
    const int kb = blockIdx.z * KC, ke = min(kb + KC, g.nz);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const double rdt = sc->rho0 * inv_dt;          // rho0 / dt
    const double kx = rdt * g.idx, ky = rdt * g.idy;
    const int i = i0 + tx, j = j0 + ty;
    const int im = wrapm(i - 1, nx), jm = wrapm(j - 1, ny);

    if (tile_uniform(g, sc)) {
        double wlo = 0.0;
        if (!(g.walls && kb == 0)) wlo = __ldg(w + ((size_t)(kb == 0 ? nz - 1 : kb - 1) * ny + j) * nx + i);
        if (g.iso) {
            // One spacing h: f = (rho0/(dt h)) [(u_i - u_{i-1}) + (v_j - v_{j-1}) + (w_k - w_{k-1})].
            // The bracket is summed exactly in 64-bit fixed point at the scale of the cell's
            // largest exponent (integer operations), leaving one conversion and one multiply
            // in FP64 (instead of six FP64 instructions).  kx = rho0/(dt h) is rescaled by
            // 2^(emax - 1080) through its exponent field.
            const long long kb_bits = __double_as_longlong(kx);
            const int ke_x = (int)((kb_bits >> 52) & 0x7FF);
            for (int k = kb; k < ke; ++k) {
                const size_t row = (size_t)k * ny;
                const size_t qc = (row + j) * nx + i;
                const double whi = (g.walls && k == nz - 1) ? 0.0 : __ldg(w + qc);
                const double uc = __ldg(u + qc), um = __ldg(u + (row + j) * nx + im);
                const double vc = __ldg(v + qc), vm = __ldg(v + (row + jm) * nx + i);
                const int emax = max(max(max(bexp(uc), bexp(um)), max(bexp(vc), bexp(vm))), max(bexp(whi), bexp(wlo)));
                const int es = ke_x + emax - 1080;
                double fv;
                if (emax < 2047 && es >= 1 && es <= 2046) {
                    const long long S = (fixe(uc, emax) - fixe(um, emax)) + (fixe(vc, emax) - fixe(vm, emax)) +
                                        (fixe(whi, emax) - fixe(wlo, emax));
                    fv = __ll2double_rn(S) * __longlong_as_double(kb_bits + ((long long)(emax - 1080) << 52));
                } else {                  // non-finite input, or a scale outside binary64: plain FP64
                    fv = kx * ((uc - um) + (vc - vm) + (whi - wlo));
                }
                f[qc] = fv;
                wlo = whi;
            }
            return;
        }
        // (rho0/dt)/dzf_k once per plane for the CTA (six FP64 instructions per cell remain)
        __shared__ double kzf[KC];
        if (tid < ke - kb) kzf[tid] = rdt * __ldg(g.idzf + kb + tid);
        __syncthreads();
        for (int k = kb; k < ke; ++k) {
            const size_t row = (size_t)k * ny;
            const size_t qc = (row + j) * nx + i;
            const double whi = (g.walls && k == nz - 1) ? 0.0 : __ldg(w + qc);
            const double du = __ldg(u + qc) - __ldg(u + (row + j) * nx + im);
            const double dv = __ldg(v + qc) - __ldg(v + (row + jm) * nx + i);
            f[qc] = fma(du, kx, fma(dv, ky, (whi - wlo) * kzf[k - kb]));
            wlo = whi;
        }
        return;
    }

    const double s = dt * sc->inv_rho0;            // dt / rho0
    const double s1 = s * c1, s2 = s * c2;         // p~ = s1 p^n - s2 p^{n-1}
    const bool two = pnm1 != nullptr;
    auto pt_at = [&](size_t q) -> double {
        const double a = s1 * __ldg(pn + q);
        return two ? fma(-s2, __ldg(pnm1 + q), a) : a;
    };
    auto fill = [&](int k, int buf) {
        for (int e = tid; e < (TY + 2) * (RX + 2); e += nthr) {
            const int bb = e / (RX + 2), aa = e - bb * (RX + 2);
            const int jj = wrapm(j0 - 1 + bb, ny), ii = wrapm(i0 - 1 + aa, nx);
            Pt[buf][bb][aa] = pt_at(((size_t)k * ny + jj) * nx + ii);
        }
    };
    // z flux through the bottom face of cell kb
    double qz_lo = 0.0;
    if (!(g.walls && kb == 0)) {
        const int km = kb == 0 ? nz - 1 : kb - 1;
        const size_t qm = ((size_t)km * ny + j) * nx + i;
        const size_t qc = ((size_t)kb * ny + j) * nx + i;
        qz_lo = fma(__ldg(bz + qm), pt_at(qc) - pt_at(qm), __ldg(w + qm));
    }
    fill(kb, kb & 1);
    for (int k = kb; k < ke; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        const bool top = g.walls && (k == nz - 1);
        if (!top) fill(k + 1 == nz ? 0 : k + 1, nxt);
        __syncthreads();
        for (int e = tid; e < TY * (RX + 1); e += nthr) {       // x faces i0-1/2 .. i0+RX-1/2
            const int b = e / (RX + 1), a = e - b * (RX + 1);
            const size_t q = ((size_t)k * ny + (j0 + b)) * nx + (wrapm(i0 - 1 + a, nx));
            QX[b][a] = fma(__ldg(bx + q), Pt[cur][b + 1][a + 1] - Pt[cur][b + 1][a], __ldg(u + q));
        }
        for (int e = tid; e < (TY + 1) * RX; e += nthr) {       // y faces j0-1/2 .. j0+TY-1/2
            const int b = e / RX, a = e - b * RX;
            const size_t q = ((size_t)k * ny + (wrapm(j0 - 1 + b, ny))) * nx + (i0 + a);
            QY[b][a] = fma(__ldg(by + q), Pt[cur][b + 1][a + 1] - Pt[cur][b][a + 1], __ldg(v + q));
        }
        const size_t qc = ((size_t)k * ny + j) * nx + i;
        double qz_hi = 0.0;
        if (!top) qz_hi = fma(__ldg(bz + qc), Pt[nxt][ty + 1][tx + 1] - Pt[cur][ty + 1][tx + 1], __ldg(w + qc));
        __syncthreads();
        const double kz = rdt * __ldg(g.idzf + k);
        f[qc] = fma(QX[ty][tx + 1] - QX[ty][tx], kx, fma(QY[ty + 1][tx] - QY[ty][tx], ky, (qz_hi - qz_lo) * kz));
        qz_lo = qz_hi;
    }
}

// --------------------------------------------------------------------- correct
// Each cell owns the faces above it: u_new = u - a (p_+ - p) + b (p~_+ - p~), a = dt/(rho0 h).
// A tile with every face coefficient zero skips p~ (same bits: the b term is +0).
template <int RX, int TY>
__global__ void __launch_bounds__(RX * TY) k_correct(const double* __restrict__ p, const double* __restrict__ pn,
                                                     const double* __restrict__ pnm1, const double* __restrict__ bx,
                                                     const double* __restrict__ by, const double* __restrict__ bz,
                                                     double* __restrict__ u, double* __restrict__ v,
                                                     double* __restrict__ w, Geo g, double c1, double c2,
                                                     double dt, const DevScalars* __restrict__ sc) {
    __shared__ double Pt[2][TY + 1][RX + 1];
    constexpr int KC = FLUPS_KC;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RX + tx, nthr = RX * TY;
    const int i0 = blockIdx.x * RX, j0 = blockIdx.y * TY;
    const int kb = blockIdx.z * KC, ke = min(kb + KC, g.nz);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const double s = dt * sc->inv_rho0;
    const double ax = s * g.idx, ay = s * g.idy;
    const int i = i0 + tx, j = j0 + ty;
    const int ie = wrapm(i + 1, nx), jn = wrapm(j + 1, ny);

    if (tile_uniform(g, sc)) {
        // -(dt/rho0)/dzc_k once per plane for the CTA (six FP64 instructions per cell remain)
        __shared__ double azc[KC];
        if (tid < ke - kb) azc[tid] = -(s * __ldg(g.idzc + kb + tid));
        __syncthreads();
        for (int k = kb; k < ke; ++k) {
            const bool top = g.walls && (k == nz - 1);
            const int kp = k + 1 == nz ? 0 : k + 1;
            const size_t qc = ((size_t)k * ny + j) * nx + i;
            const double pc = __ldg(p + qc);
            const double pe = __ldg(p + ((size_t)k * ny + j) * nx + ie);
            const double pnb = __ldg(p + ((size_t)k * ny + jn) * nx + i);
            u[qc] = fma(-ax, pe - pc, u[qc]);
            v[qc] = fma(-ay, pnb - pc, v[qc]);
            if (top) {
                w[qc] = 0.0;
            } else {
                const double pt = __ldg(p + ((size_t)kp * ny + j) * nx + i);
                w[qc] = fma(azc[k - kb], pt - pc, w[qc]);
            }
        }
        return;
    }

    const double s1 = s * c1, s2 = s * c2;
    const bool two = pnm1 != nullptr;
    auto pt_at = [&](size_t q) -> double {
        const double a = s1 * __ldg(pn + q);
        return two ? fma(-s2, __ldg(pnm1 + q), a) : a;
    };
    auto fill = [&](int k, int buf) {
        for (int e = tid; e < (TY + 1) * (RX + 1); e += nthr) {
            const int bb = e / (RX + 1), aa = e - bb * (RX + 1);
            const int jj = wrapm(j0 + bb, ny), ii = wrapm(i0 + aa, nx);
            Pt[buf][bb][aa] = pt_at(((size_t)k * ny + jj) * nx + ii);
        }
    };
    fill(kb, kb & 1);
    for (int k = kb; k < ke; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        const bool top = g.walls && (k == nz - 1);
        const int kp = k + 1 == nz ? 0 : k + 1;
        if (!top) fill(kp, nxt);
        __syncthreads();
        const size_t qc = ((size_t)k * ny + j) * nx + i;
        const double pc = __ldg(p + qc);
        const double pe = __ldg(p + ((size_t)k * ny + j) * nx + ie);
        const double pnb = __ldg(p + ((size_t)k * ny + jn) * nx + i);
        const double ptc = Pt[cur][ty][tx];
        u[qc] = fma(-ax, pe - pc, fma(__ldg(bx + qc), Pt[cur][ty][tx + 1] - ptc, u[qc]));
        v[qc] = fma(-ay, pnb - pc, fma(__ldg(by + qc), Pt[cur][ty + 1][tx] - ptc, v[qc]));
        if (top) {
            w[qc] = 0.0;
        } else {
            const double pt = __ldg(p + ((size_t)kp * ny + j) * nx + i);
            const double az = s * __ldg(g.idzc + k);
            w[qc] = fma(-az, pt - pc, fma(__ldg(bz + qc), Pt[nxt][ty][tx] - ptc, w[qc]));
        }
        __syncthreads();
    }
}

// ------------------------------------------------- FP64 residual norm (reporting)
// part[3b+0] = sum dzf f, [3b+1] = sum (f - m)^2 ... computed in two kernels:
// pass 0: sum dzf f, sum f^2, sum f; pass 1 (needs mean_f): sum r^2 with r = f - m - L p.
__global__ void __launch_bounds__(256) k_res64(const double* __restrict__ f, const double* __restrict__ p, Geo g,
                                               const DevScalars* __restrict__ sc, int pass,
                                               double* __restrict__ part) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double a = 0.0, b = 0.0, c = 0.0;
    const double mf = pass == 1 ? sc->mean_f : 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % g.nx);
        const size_t rr = q / g.nx;
        const int j = (int)(rr % g.ny), k = (int)(rr / g.ny);
        const double fv = f[q];
        if (pass == 0) {
            a = fma(fv, g.dzf[k], a);
            b = fma(fv, fv, b);
            c += fv;
        } else {
            const size_t row = rr * g.nx;
            const double pc = p[q];
            const double pw = p[row + (wrapm(i - 1, g.nx))], pe = p[row + (wrapm(i + 1, g.nx))];
            const double ps = p[((size_t)k * g.ny + (wrapm(j - 1, g.ny))) * g.nx + i];
            const double pnn = p[((size_t)k * g.ny + (wrapm(j + 1, g.ny))) * g.nx + i];
            int km, kp;
            if (g.walls) { km = k > 0 ? k - 1 : 0; kp = k < g.nz - 1 ? k + 1 : g.nz - 1; }
            else { km = (k - 1 + g.nz) % g.nz; kp = (k + 1) % g.nz; }
            const double pb = p[((size_t)km * g.ny + j) * g.nx + i], pt = p[((size_t)kp * g.ny + j) * g.nx + i];
            const double lp = g.sx * (pw + pe - 2.0 * pc) + g.sy * (ps + pnn - 2.0 * pc) + g.az[k] * (pb - pc) +
                              g.cz[k] * (pt - pc);
            const double r = (fv - mf) - lp;
            b = fma(r, r, b);
        }
    }
    __shared__ double red[3][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][wid] = a; red[1][wid] = b; red[2][wid] = c; }
    __syncthreads();
    if (wid == 0) {
        a = lane < nw ? red[0][lane] : 0.0;
        b = lane < nw ? red[1][lane] : 0.0;
        c = lane < nw ? red[2][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
            c += __shfl_down_sync(0xffffffffu, c, o);
        }
        if (lane == 0) { part[3 * blockIdx.x] = a; part[3 * blockIdx.x + 1] = b; part[3 * blockIdx.x + 2] = c; }
    }
}

__global__ void k_res64_finalize(const double* __restrict__ part, int nblk, DevScalars* sc, int pass, double nrm_w,
                                 double npts) {
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = 0; q < nblk; ++q) { a += part[3 * q]; b += part[3 * q + 1]; c += part[3 * q + 2]; }
    if (pass == 0) {
        const double m = a * nrm_w;
        sc->mean_f = m;
        sc->f2 = b - 2.0 * m * c + npts * m * m;
    } else {
        sc->r2 = b;
    }
}

template <int RX>
void run_rhs(flups_plan P, const double* u, const double* v, const double* w, const double* pn,
             const double* pnm1, double c1, double c2, double dt, double* f, const Geo& g) {
    constexpr int TY = FLUPS_TY;
    dim3 grid(g.tnx, g.tny, g.tnz);
    flups_prof_begin(P, FK_RHS);
    k_rhs<RX, TY><<<grid, dim3(RX, TY), 0, P->stream>>>(u, v, w, pn, pnm1, P->bx, P->by, P->bz, f, g, c1, c2, dt,
                                                         1.0 / dt, P->sc);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
}

template <int RX>
void run_correct(flups_plan P, const double* p, const double* pn, const double* pnm1, double c1, double c2,
                 double dt, double* u, double* v, double* w, const Geo& g) {
    constexpr int TY = FLUPS_TY;
    dim3 grid(g.tnx, g.tny, g.tnz);
    flups_prof_begin(P, FK_CORRECT);
    k_correct<RX, TY><<<grid, dim3(RX, TY), 0, P->stream>>>(p, pn, pnm1, P->bx, P->by, P->bz, u, v, w, g, c1, c2,
                                                             dt, P->sc);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
}

}  // namespace

cudaError_t launch_set_density(flups_plan P, const double* rho, double rho0) {
    const Geo g = plan_geo(P);
    const int ntiles = g.tnx * g.tny * g.tnz;
    dim3 tgrid(g.tnx, g.tny, g.tnz);
    long long* part = reinterpret_cast<long long*>(P->part);
    flups_prof_begin(P, FK_RHO_MINMAX);
    if (g.rx == 32) k_rho_tiles<32><<<tgrid, dim3(32, FLUPS_TY), 0, P->stream>>>(rho, g, P->trange, part);
    else if (g.rx == 16) k_rho_tiles<16><<<tgrid, dim3(16, FLUPS_TY), 0, P->stream>>>(rho, g, P->trange, part);
    else k_rho_tiles<8><<<tgrid, dim3(8, FLUPS_TY), 0, P->stream>>>(rho, g, P->trange, part);
    flups_prof_end(P);
    flups_prof_begin(P, FK_TILE_FLAGS);
    k_rho_finalize<<<1, 1024, 0, P->stream>>>(part, ntiles, P->sc, rho0, g.idx, g.idy);
    flups_prof_end(P);
    flups_prof_begin(P, FK_FACE_COEFFS);
    if (g.rx == 32) k_face_coeffs<32><<<tgrid, dim3(32, FLUPS_TY), 0, P->stream>>>(rho, P->bx, P->by, P->bz, g, P->sc);
    else if (g.rx == 16) k_face_coeffs<16><<<tgrid, dim3(16, FLUPS_TY), 0, P->stream>>>(rho, P->bx, P->by, P->bz, g, P->sc);
    else k_face_coeffs<8><<<tgrid, dim3(8, FLUPS_TY), 0, P->stream>>>(rho, P->bx, P->by, P->bz, g, P->sc);
    flups_prof_end(P);
    FLUPS_COUNT(P, 3);
    return cudaGetLastError();
}

cudaError_t launch_rhs(flups_plan P, const double* u, const double* v, const double* w, const double* pn,
                       const double* pnm1, double c1, double c2, double dt, double* f) {
    const Geo g = plan_geo(P);
    if (g.rx == 32) run_rhs<32>(P, u, v, w, pn, pnm1, c1, c2, dt, f, g);
    else if (g.rx == 16) run_rhs<16>(P, u, v, w, pn, pnm1, c1, c2, dt, f, g);
    else run_rhs<8>(P, u, v, w, pn, pnm1, c1, c2, dt, f, g);
    return cudaGetLastError();
}

cudaError_t launch_correct(flups_plan P, const double* p, const double* pn, const double* pnm1, double c1,
                           double c2, double dt, double* u, double* v, double* w) {
    const Geo g = plan_geo(P);
    if (g.rx == 32) run_correct<32>(P, p, pn, pnm1, c1, c2, dt, u, v, w, g);
    else if (g.rx == 16) run_correct<16>(P, p, pn, pnm1, c1, c2, dt, u, v, w, g);
    else run_correct<8>(P, p, pn, pnm1, c1, c2, dt, u, v, w, g);
    return cudaGetLastError();
}

cudaError_t launch_residual64_norm(flups_plan P, const double* f, const double* p) {
    const Geo g = plan_geo(P);
    const int nblk = 1024;
    flups_prof_begin(P, FK_RES64);
    k_res64<<<nblk, 256, 0, P->stream>>>(f, p, g, P->sc, 0, P->part);
    k_res64_finalize<<<1, 32, 0, P->stream>>>(P->part, nblk, P->sc, 0, 1.0 / ((double)P->nx * P->ny * P->sum_dzf),
                                              (double)P->npts);
    k_res64<<<nblk, 256, 0, P->stream>>>(f, p, g, P->sc, 1, P->part);
    k_res64_finalize<<<1, 32, 0, P->stream>>>(P->part, nblk, P->sc, 1, 0.0, 0.0);
    flups_prof_end(P);
    FLUPS_COUNT(P, 4);
    return cudaGetLastError();
}
