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
__device__ __forceinline__ double recip64(double s) {
    const float sf = __double2float_rn(s);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(sf));
    double y = (double)yf;
    double e = fma(-s, y, 1.0);
    y = fma(y, e, y);
    e = fma(-s, y, 1.0);
    return fma(y, e, y);
}

// Valid densities: finite and within [1e-30, 1e30] (so the FP32 seed above is normal).
// Positive doubles order like their bit patterns, so the test is two integer compares.
__device__ __forceinline__ bool rho_bad(double r) {
    const long long b = __double_as_longlong(r);
    return b < 0x39B4484BFEEBC2A0LL || b > 0x46293E5939A08CEALL;   // 1e-30, 1e30
}

__global__ void k_rho_minmax(const double* __restrict__ rho, size_t n, long long* __restrict__ part) {
    long long mn = 0x7FFFFFFFFFFFFFFFLL;
    int bad = 0;
    // four 16-byte loads in flight per thread (n is even: nx is a power of two >= 8)
    const double2* r2 = reinterpret_cast<const double2*>(rho);
    const size_t n2 = n / 2, stride = (size_t)gridDim.x * blockDim.x;
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n2; i += 4 * stride) {
        double2 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __ldg(r2 + i + q * stride);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long a = __double_as_longlong(v[q].x), b = __double_as_longlong(v[q].y);
            mn = a < mn ? a : mn;
            mn = b < mn ? b : mn;
            bad |= rho_bad(v[q].x) | rho_bad(v[q].y);
        }
    }
    for (; i < n2; i += stride) {
        const double2 v = __ldg(r2 + i);
        const long long a = __double_as_longlong(v.x), b = __double_as_longlong(v.y);
        mn = a < mn ? a : mn;
        mn = b < mn ? b : mn;
        bad |= rho_bad(v.x) | rho_bad(v.y);
    }
    __shared__ long long smn[32];
    __shared__ int sbad[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_down_sync(0xffffffffu, mn, o);
        mn = t < mn ? t : mn;
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { smn[wid] = mn; sbad[wid] = bad; }
    __syncthreads();
    if (wid == 0) {
        mn = lane < nw ? smn[lane] : 0x7FFFFFFFFFFFFFFFLL;
        bad = lane < nw ? sbad[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long t = __shfl_down_sync(0xffffffffu, mn, o);
            mn = t < mn ? t : mn;
            bad |= __shfl_down_sync(0xffffffffu, bad, o);
        }
        if (lane == 0) { part[2 * blockIdx.x] = mn; part[2 * blockIdx.x + 1] = bad; }
    }
}

__global__ void k_rho_finalize(const long long* __restrict__ part, int nblk, DevScalars* sc, double rho0_user,
                               double idx, double idy) {
    if (threadIdx.x != 0) return;
    long long mn = 0x7FFFFFFFFFFFFFFFLL;
    int bad = 0;
    for (int i = 0; i < nblk; ++i) {
        mn = part[2 * i] < mn ? part[2 * i] : mn;
        bad |= (int)part[2 * i + 1];
    }
    const double r0 = rho0_user > 0.0 ? rho0_user : __longlong_as_double(mn);
    sc->rho0 = r0;
    sc->inv_rho0 = 1.0 / r0;
    sc->m2r0 = -2.0 * r0;
    sc->m2r0_dx = -2.0 * r0 * idx;
    sc->m2r0_dy = -2.0 * r0 * idy;
    sc->bad_rho = bad;
}

// Tile flags: a face whose two cells both hold exactly rho0 has (1 - rho0/rho_f) = 0; the
// test runs on the bit patterns, without FP64 instructions.  Every stencil tile whose CTA
// reads a nonzero coefficient is flagged: the tile that owns the cell, and the tile above
// it in x, y or z when the cell's face is that tile's lower boundary face.
__global__ void __launch_bounds__(256) k_tile_flags(const double* __restrict__ rho, Geo g,
                                                    const DevScalars* __restrict__ sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    const bool act = i < g.nx;
    const long long b0 = __double_as_longlong(sc->rho0);
    long long bc_ = b0, be = b0, bn = b0, bt = b0;
    bool top_wall = g.walls && k == g.nz - 1;
    if (act) {
        const size_t idx = ((size_t)k * g.ny + j) * g.nx + i;
        bc_ = __double_as_longlong(__ldg(rho + idx));
        be = __double_as_longlong(__ldg(rho + ((size_t)k * g.ny + j) * g.nx + (wrapm(i + 1, g.nx))));
        bn = __double_as_longlong(__ldg(rho + ((size_t)k * g.ny + (wrapm(j + 1, g.ny))) * g.nx + i));
        const int kp = g.walls ? (k + 1 < g.nz ? k + 1 : k) : (k + 1 == g.nz ? 0 : k + 1);
        bt = __double_as_longlong(__ldg(rho + ((size_t)kp * g.ny + j) * g.nx + i));
    }
    const bool cz0 = bc_ == b0;
    const bool nzx = act && !(cz0 && be == b0), nzy = act && !(cz0 && bn == b0);
    const bool nzz = act && !(cz0 && bt == b0) && !top_wall;
    const int tx = i >> g.lgrx, ty = j / FLUPS_TY, tz = k / FLUPS_KC;
    const int txp = (tx + 1 == g.tnx) ? 0 : tx + 1;
    const int typ = (ty + 1 == g.tny) ? 0 : ty + 1;
    const int tzp = (tz + 1 == g.tnz) ? 0 : tz + 1;
    const bool last_x = act && ((i & (g.rx - 1)) == g.rx - 1), last_y = (j % FLUPS_TY) == FLUPS_TY - 1;
    const bool last_z = (k % FLUPS_KC) == FLUPS_KC - 1 || k == g.nz - 1;
    auto tile = [&](int a, int b, int c) { return (size_t)(c * g.tny + b) * g.tnx + a; };
    if (g.rx == 32) {
        // the 32 lanes of a warp are the 32 columns of one tile row
        const unsigned any = __ballot_sync(0xffffffffu, nzx || nzy || nzz);
        const unsigned anyy = __ballot_sync(0xffffffffu, nzy);
        const unsigned anyz = __ballot_sync(0xffffffffu, nzz);
        if ((threadIdx.x & 31) == 0 && act) {
            if (any) atomicOr(g.tflags + tile(tx, ty, tz), 1u);
            if (anyy && last_y) atomicOr(g.tflags + tile(tx, typ, tz), 1u);
            if (anyz && last_z) atomicOr(g.tflags + tile(tx, ty, tzp), 1u);
        }
        if (nzx && last_x) atomicOr(g.tflags + tile(txp, ty, tz), 1u);
    } else if (act) {
        if (nzx || nzy || nzz) atomicOr(g.tflags + tile(tx, ty, tz), 1u);
        if (nzx && last_x) atomicOr(g.tflags + tile(txp, ty, tz), 1u);
        if (nzy && last_y) atomicOr(g.tflags + tile(tx, typ, tz), 1u);
        if (nzz && last_z) atomicOr(g.tflags + tile(tx, ty, tzp), 1u);
    }
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
    if (g.tflags[(blockIdx.z * g.tny + blockIdx.y) * g.tnx + blockIdx.x] == 0) return;
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

    if (g.tflags[(blockIdx.z * g.tny + blockIdx.y) * g.tnx + blockIdx.x] == 0) {
        double wlo = 0.0;
        if (!(g.walls && kb == 0)) wlo = __ldg(w + ((size_t)(kb == 0 ? nz - 1 : kb - 1) * ny + j) * nx + i);
        for (int k = kb; k < ke; ++k) {
            const size_t row = (size_t)k * ny;
            const size_t qc = (row + j) * nx + i;
            const double whi = (g.walls && k == nz - 1) ? 0.0 : __ldg(w + qc);
            const double du = __ldg(u + qc) - __ldg(u + (row + j) * nx + im);
            const double dv = __ldg(v + qc) - __ldg(v + (row + jm) * nx + i);
            f[qc] = fma(du, kx, fma(dv, ky, (whi - wlo) * (rdt * __ldg(g.idzf + k))));
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

    if (g.tflags[(blockIdx.z * g.tny + blockIdx.y) * g.tnx + blockIdx.x] == 0) {
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
                w[qc] = fma(-(s * __ldg(g.idzc + k)), pt - pc, w[qc]);
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
    const int nblk = 1024;
    flups_prof_begin(P, FK_RHO_MINMAX);
    k_rho_minmax<<<nblk, 256, 0, P->stream>>>(rho, P->npts, reinterpret_cast<long long*>(P->part));
    k_rho_finalize<<<1, 32, 0, P->stream>>>(reinterpret_cast<const long long*>(P->part), nblk, P->sc, rho0, g.idx,
                                            g.idy);
    flups_prof_end(P);
    cudaMemsetAsync(P->tflags, 0, (size_t)g.tnx * g.tny * g.tnz * sizeof(unsigned int), P->stream);
    dim3 grid((g.nx + 255) / 256, g.ny, g.nz);
    flups_prof_begin(P, FK_TILE_FLAGS);
    k_tile_flags<<<grid, 256, 0, P->stream>>>(rho, g, P->sc);
    flups_prof_end(P);
    flups_prof_begin(P, FK_FACE_COEFFS);
    dim3 tgrid(g.tnx, g.tny, g.tnz);
    if (g.rx == 32) k_face_coeffs<32><<<tgrid, dim3(32, FLUPS_TY), 0, P->stream>>>(rho, P->bx, P->by, P->bz, g, P->sc);
    else if (g.rx == 16) k_face_coeffs<16><<<tgrid, dim3(16, FLUPS_TY), 0, P->stream>>>(rho, P->bx, P->by, P->bz, g, P->sc);
    else k_face_coeffs<8><<<tgrid, dim3(8, FLUPS_TY), 0, P->stream>>>(rho, P->bx, P->by, P->bz, g, P->sc);
    flups_prof_end(P);
    FLUPS_COUNT(P, 4);
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
