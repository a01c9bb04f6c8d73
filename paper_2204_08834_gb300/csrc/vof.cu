// vof.cu - the volume-of-fluid step: MTHINC reconstruction and directional-split advection of
// the volume fraction phi (FluTAS Sec. 3.1, Eqs. phi_split and vof_corr_step; Appendix A) on a
// triply periodic grid.
//
// H(x~) = (1 + tanh(beta (T(x~) + d))) / 2 in the cell's local coordinates x~ in [0, 1]^3, T the
// quadratic of App. A.1 built from the Youngs normal n and K = grad n, linear along the case
// direction p (the largest normal component), d = d_th normalising the cell integral of H to phi
// (integral exact along p, two-point Gauss-Legendre along the other two directions).
//
// Per split direction s, in the order x, y, z:
//   k_vof_rec    per cell: case p, the coefficients of T in the case's frame and d_th (FP32),
//                or a uniform mark (phi <= 1e-8, phi >= 1 - 1e-8, zero gradient).  The case
//                decision is an integer taken from floating point: it is taken on the Youngs
//                gradient summed with explicitly rounded binary32 operations in the order of the
//                definition, the same operations a binary32 evaluation of the formula performs.
//                An 8^3 tile of cells shares its 9^3 corner gradients through shared memory.
//   k_vof_flux   per face i+1/2 along s: the integral of H of the upwind cell over the box swept
//                in dt (exact along the cell's p, Gauss over the other two intervals), FP32 (the
//                swept fraction too), stored as one FP64 number per face; for a uniform upwind
//                cell phi u dt / h in FP64.
//   k_vof_update phi^p = (phi^s - (F_{i+1/2} - F_{i-1/2})) / (1 - dt/h (u_{i+1/2} - u_{i-1/2})),
//                FP64 (the division as a product with a Newton-refined reciprocal).
// then k_vof_final: phi^{n+1} = phi^z - sum_p dt/h_p phi^p (u_{i+1/2} - u_{i-1/2})_p, FP64.
// Each face flux is one stored number used by both cells beside the face and the updates run in
// FP64, so sum(phi) is conserved to FP64 rounding whatever the rounding of the FP32 fluxes.
#include <cmath>

#include "flups_impl.cuh"
#include "fp_bits.cuh"

namespace {

constexpr double kEpsUniform = 1e-8;
constexpr int VT = 8;            // reconstruction tile edge (cells)
constexpr int VC = VT + 1;       // corner grid edge of a tile
constexpr int VP = VT + 2;       // phi tile edge with its one-cell halo

struct VofGeo {
    int nx, ny, nz;
    double dt;
    double h[3];       // dx, dy, dz
    double c[3];       // dt / dx, dt / dy, dt / dz
    float cf[3];       // the same in FP32 (the flux pass's swept fractions)
    float beta;
};

// 1/x in FP64 from the binary32 reciprocal refined by two Newton steps (each doubles the
// correct bits: 24 -> 48 -> beyond 53): four FMAs on GB300's narrow FP64 pipe (the conversions
// by integer operations), against an IEEE division's longer sequence; within one unit in the
// last place of 1/x.
__device__ __forceinline__ double rcp64(double x) {
    double r = f2d_bits(1.0f / d2f_bits(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// 1/x by the hardware reciprocal approximation (about 2^-23 relative, FP32 rounding size).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The cell record: case p (-1: uniform) and T = q1 x1^2 + q2 x2^2 + r x1 x2 + Lp xp + L1 x1 + L2 x2
// in the case frame (x1, x2 the two other directions in increasing order), d = d_th.
struct __align__(16) VofRec {
    float p, q1, q2, r, Lp, L1, L2, d;
};

__device__ __forceinline__ float gval(const VofRec& R, float t1, float t2) {
    return R.q1 * t1 * t1 + R.q2 * t2 * t2 + R.r * t1 * t2 + R.L1 * t1 + R.L2 * t2;
}

// softplus(y) = ln(1 + e^y) and logistic(y) = 1/(1 + e^-y) from one exponential (y clamped to
// +-80, where both have reached their limits in FP32): for y > 15 softplus is y to FP32
// precision, for small e^y it is e^y (1 - e^y / 2).
__device__ __forceinline__ void sp_sig(float y, float& sp, float& sg) {
    const float e = __expf(fminf(fmaxf(y, -80.f), 80.f));
    const float one = 1.f + e;
    sp = y > 15.f ? y : (e < 1e-3f ? e * (1.f - 0.5f * e) : __logf(one));
    sg = e * rcp_approx(one);
}

// Volume equation of d (App. A.1.2) for one cell: W(d) = the two-point Gauss mean over the unit
// square of the exact line integrals along p of H (or, MINOR, of 1 - H: the arguments negated),
// W = sg sum_q [softplus(y1_q) - softplus(y0_q)] / (4 tb a) with y1 = tb (a + g_q + d),
// y0 = tb (g_q + d), tb = 2 beta, sg = -1 for MINOR; dW/dd = sum_q [logistic(y1) - logistic(y0)]
// / (4 a).  gq: T at the four Gauss nodes (x~_p = 0).
template <bool MINOR>
__device__ __forceinline__ void volume_eq(const float* gq, float a, float tb, float d, float& W, float& dW) {
    float sw = 0.f, sd = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float y1 = tb * (a + gq[q] + d), y0 = tb * (gq[q] + d);
        if (MINOR) { y1 = -y1; y0 = -y0; }
        float p1, s1, p0, s0;
        sp_sig(y1, p1, s1);
        sp_sig(y0, p0, s0);
        sw += p1 - p0;
        sd += s1 - s0;
    }
    const float ia = rcp_approx(a);
    W = (MINOR ? -0.25f : 0.25f) * sw * ia / tb;
    dW = 0.25f * sd * ia;
}

// d_th by safeguarded Newton on ln W(d) = ln target (W the volume of the cell's minority phase,
// monotone in d).  ln W is concave in d (an integral of log-concave logistic factors), so Newton
// overshoots at most once and then converges from one side; a bracket [lo, hi] on which
// W - target changes sign takes over when a step leaves it.  Start: for a small minority volume
// the limit W ~ exp(+-2 beta d) M (softplus(y) ~ e^y), M the Gauss mean of the exact line
// integrals of exp(+-2 beta T); otherwise where T + d vanishes at the cell centre.
template <bool MINOR>
__device__ float solve_d(const VofRec& R, float beta, float target, float lo, float hi) {
    constexpr float g0 = 0.21132486540518712f, g1 = 0.78867513459481288f;   // (1 -+ 1/sqrt 3) / 2
    float gq[4];
    gq[0] = gval(R, g0, g0);
    gq[1] = gval(R, g0, g1);
    gq[2] = gval(R, g1, g0);
    gq[3] = gval(R, g1, g1);
    const float a = R.Lp, tb = 2.f * beta;
    float d;
    if (target < 0.1f) {
        const float ts = MINOR ? -tb : tb;
        float Mq = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) Mq += __expf(ts * (a + gq[q])) - __expf(ts * gq[q]);
        d = (__logf(target) - __logf(0.25f * Mq / (ts * a))) / ts;
        if (!(d == d)) d = 0.5f * (lo + hi);
    } else {
        d = -(gval(R, 0.5f, 0.5f) + 0.5f * a);
    }
    d = fminf(fmaxf(d, lo), hi);
    const float lt = __logf(target);
    for (int it = 0; it < 40; ++it) {
        float W, dW;
        volume_eq<MINOR>(gq, a, tb, d, W, dW);
        const bool up = MINOR ? (W > target) : (W < target);     // the root lies above d
        if (up) lo = d; else hi = d;
        float dn;
        if (W > 0.f && dW != 0.f) dn = d - (__logf(W) - lt) * W * rcp_approx(dW);
        else dn = 0.5f * (lo + hi);
        if (!(dn > lo && dn < hi)) dn = 0.5f * (lo + hi);
        const float step = fabsf(dn - d);
        d = dn;
        if (step <= 2e-7f * (1.f + fabsf(d)) || hi - lo <= 2e-7f * (1.f + fabsf(d))) break;
    }
    return d;
}

// Reconstruction of an 8^3 tile (512 threads).  Shared memory: phi of the tile and its halo
// rounded to binary32, and the 9^3 corner gradients (each component the difference across the
// corner averaged over its four cell pairs) with their normalised copies.  The gradient sums
// use explicitly rounded binary32 operations in a fixed order, the order of the definition, so
// the case decision and the zero-gradient test are bit for bit those of a binary32 evaluation
// of the same formula.
__global__ void __launch_bounds__(512) k_vof_rec(const double* __restrict__ phi, VofRec* __restrict__ rec, VofGeo g) {
    __shared__ float ph[VP][VP][VP];
    __shared__ float mc[3][VC][VC][VC];
    __shared__ float nc[3][VC][VC][VC];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * VT, y0 = blockIdx.y * VT, z0 = blockIdx.z * VT;
    for (int q = tid; q < VP * VP * VP; q += blockDim.x) {
        const int a = q % VP, b = (q / VP) % VP, c = q / (VP * VP);
        const int gx = wrapi(x0 - 1 + a, g.nx), gy = wrapi(y0 - 1 + b, g.ny), gz = wrapi(z0 - 1 + c, g.nz);
        ph[c][b][a] = __double2float_rn(__ldg(&phi[((size_t)gz * g.ny + gy) * g.nx + gx]));
    }
    __syncthreads();
    // corner (ci, cj, ck): between cells ci-1, ci (tile coordinates), i.e. lower cell at ph index
    // (ci, cj, ck); per component d = phi(upper) - phi(lower) across the corner at the four
    // positions of the two other directions, summed ((d00 + d10) + d01) + d11 with "1" the
    // shift along the first and then the second other direction, times 1/4
    for (int q = tid; q < VC * VC * VC; q += blockDim.x) {
        const int ci = q % VC, cj = (q / VC) % VC, ck = q / (VC * VC);
        float gx, gy, gz;
        {
            const float d00 = __fsub_rn(ph[ck][cj][ci + 1], ph[ck][cj][ci]);
            const float d10 = __fsub_rn(ph[ck][cj + 1][ci + 1], ph[ck][cj + 1][ci]);
            const float d01 = __fsub_rn(ph[ck + 1][cj][ci + 1], ph[ck + 1][cj][ci]);
            const float d11 = __fsub_rn(ph[ck + 1][cj + 1][ci + 1], ph[ck + 1][cj + 1][ci]);
            gx = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(__fadd_rn(d00, d10), d01), d11));
        }
        {
            const float d00 = __fsub_rn(ph[ck][cj + 1][ci], ph[ck][cj][ci]);
            const float d10 = __fsub_rn(ph[ck][cj + 1][ci + 1], ph[ck][cj][ci + 1]);
            const float d01 = __fsub_rn(ph[ck + 1][cj + 1][ci], ph[ck + 1][cj][ci]);
            const float d11 = __fsub_rn(ph[ck + 1][cj + 1][ci + 1], ph[ck + 1][cj][ci + 1]);
            gy = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(__fadd_rn(d00, d10), d01), d11));
        }
        {
            const float d00 = __fsub_rn(ph[ck + 1][cj][ci], ph[ck][cj][ci]);
            const float d10 = __fsub_rn(ph[ck + 1][cj][ci + 1], ph[ck][cj][ci + 1]);
            const float d01 = __fsub_rn(ph[ck + 1][cj + 1][ci], ph[ck][cj + 1][ci]);
            const float d11 = __fsub_rn(ph[ck + 1][cj + 1][ci + 1], ph[ck][cj + 1][ci + 1]);
            gz = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(__fadd_rn(d00, d10), d01), d11));
        }
        mc[0][ck][cj][ci] = gx;
        mc[1][ck][cj][ci] = gy;
        mc[2][ck][cj][ci] = gz;
        const float nn = sqrtf(gx * gx + gy * gy + gz * gz);
        const float inv = nn > 0.f ? 1.f / nn : 0.f;
        nc[0][ck][cj][ci] = gx * inv;
        nc[1][ck][cj][ci] = gy * inv;
        nc[2][ck][cj][ci] = gz * inv;
    }
    __syncthreads();
    const int i = tid & 7, j = (tid >> 3) & 7, k = tid >> 6;
    const size_t cell = ((size_t)(z0 + k) * g.ny + (y0 + j)) * g.nx + (x0 + i);
    const double ph0 = __ldg(&phi[cell]);
    // cell gradient: its eight corners (corner indices i, i+1 etc.), summed as
    // ((mc(i) + mc(i-1)) over y, then over z), times 1/8
    float m[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float A11 = __fadd_rn(mc[a][k + 1][j + 1][i + 1], mc[a][k + 1][j + 1][i]);
        const float A01 = __fadd_rn(mc[a][k + 1][j][i + 1], mc[a][k + 1][j][i]);
        const float A10 = __fadd_rn(mc[a][k][j + 1][i + 1], mc[a][k][j + 1][i]);
        const float A00 = __fadd_rn(mc[a][k][j][i + 1], mc[a][k][j][i]);
        m[a] = __fmul_rn(__fadd_rn(__fadd_rn(A11, A01), __fadd_rn(A10, A00)), 0.125f);
    }
    VofRec R;
    const bool zero_grad = m[0] == 0.f && m[1] == 0.f && m[2] == 0.f;
    if (ph0 <= kEpsUniform || ph0 >= 1.0 - kEpsUniform || zero_grad) {
        R.p = -1.f; R.q1 = R.q2 = R.r = R.Lp = R.L1 = R.L2 = R.d = 0.f;
        rec[cell] = R;
        return;
    }
    const float amx = fabsf(m[0]), amy = fabsf(m[1]), amz = fabsf(m[2]);
    const int p = (amx >= amy && amx >= amz) ? 0 : (amy >= amz ? 1 : 2);
    const int o1 = p == 0 ? 1 : 0, o2 = p == 2 ? 1 : 2;
    float n[3];
    {
        const float inv = 1.f / sqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        n[0] = m[0] * inv; n[1] = m[1] * inv; n[2] = m[2] * inv;
    }
    // d n_b / d x~_a: corner normals at the cell's upper a side minus lower, over four corners
    float dn[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                sx += nc[b][k + u][j + v][i + 1] - nc[b][k + u][j + v][i];
                sy += nc[b][k + u][j + 1][i + v] - nc[b][k + u][j][i + v];
                sz += nc[b][k + 1][j + u][i + v] - nc[b][k][j + u][i + v];
            }
        dn[0][b] = 0.25f * sx;
        dn[1][b] = 0.25f * sy;
        dn[2][b] = 0.25f * sz;
    }
    auto K = [&](int a, int b) { return 0.5f * (dn[a][b] + dn[b][a]); };
    R.p = (float)p;
    R.q1 = 0.5f * K(o1, o1);
    R.q2 = 0.5f * K(o2, o2);
    R.r = K(o1, o2);
    R.Lp = n[p];
    R.L1 = n[o1] - 0.5f * (K(o1, o1) + K(o1, o2));
    R.L2 = n[o2] - 0.5f * (K(o2, o2) + K(o1, o2));
    const float tmax = fabsf(R.q1) + fabsf(R.q2) + fabsf(R.r) + fabsf(R.Lp) + fabsf(R.L1) + fabsf(R.L2);
    const float lo = -tmax - 40.f / g.beta, hi = tmax + 40.f / g.beta;
    R.d = ph0 <= 0.5 ? solve_d<false>(R, g.beta, (float)ph0, lo, hi)
                     : solve_d<true>(R, g.beta, (float)(1.0 - ph0), lo, hi);
    rec[cell] = R;
}

// Integral of H of a cell record over the box [lo_a, hi_a] (case frame: along p exact over
// [lop, hip], two-point Gauss over [lo1, hi1] x [lo2, hi2]).
__device__ __forceinline__ float box_int(const VofRec& R, float beta, float lop, float hip, float lo1, float hi1,
                                         float lo2, float hi2) {
    constexpr float g0 = 0.21132486540518712f, g1 = 0.78867513459481288f;
    const float gs[2] = {g0, g1};
    const float tb = 2.f * beta;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float t1 = lo1 + (hi1 - lo1) * gs[i], t2 = lo2 + (hi2 - lo2) * gs[j];
            const float c = gval(R, t1, t2) + R.d;
            float p1, s1, p0, s0;
            sp_sig(tb * (R.Lp * hip + c), p1, s1);
            sp_sig(tb * (R.Lp * lop + c), p0, s0);
            acc += p1 - p0;
        }
    return 0.25f * (hi1 - lo1) * (hi2 - lo2) * acc / (tb * R.Lp);
}

// The per-cell kernels run on the reconstruction's grid: an 8^3 tile per CTA, thread
// (tid & 7, (tid >> 3) & 7, tid >> 6) the cell (i, j, k) of the tile, so no index is divided.
__device__ __forceinline__ void tile_cell(int& ix, int& iy, int& iz) {
    const int t = threadIdx.x;
    ix = blockIdx.x * VT + (t & 7);
    iy = blockIdx.y * VT + ((t >> 3) & 7);
    iz = blockIdx.z * VT + (t >> 6);
}

__global__ void __launch_bounds__(512) k_vof_flux(const double* __restrict__ phi, const VofRec* __restrict__ rec,
                                                  const double* __restrict__ vel, double* __restrict__ F, VofGeo g,
                                                  int s, int* __restrict__ bad) {
    int ix, iy, iz;
    tile_cell(ix, iy, iz);
    const size_t cell = ((size_t)iz * g.ny + iy) * g.nx + ix;
    // swept fraction c = u dt / h in FP32 (binary64 -> binary32 by integer operations: the flux of
    // an interface cell is an FP32 quantity, and its path then runs nothing on the narrow FP64
    // pipe); the CFL test in FP32 too, so a |c| within FP32 rounding above 1 passes as 1
    const float c = d2f_bits(__ldg(&vel[cell])) * (s == 0 ? g.cf[0] : (s == 1 ? g.cf[1] : g.cf[2]));
    if (!(fabsf(c) <= 1.f)) {              // CFL above 1 (or not finite) along the split direction
        atomicExch(bad, 1);
        F[cell] = 0.0;
        return;
    }
    size_t up = cell;
    if (c < 0.f) {                          // the cell above the face
        int jx = ix, jy = iy, jz = iz;
        if (s == 0) jx = ix + 1 == g.nx ? 0 : ix + 1;
        else if (s == 1) jy = iy + 1 == g.ny ? 0 : iy + 1;
        else jz = iz + 1 == g.nz ? 0 : iz + 1;
        up = ((size_t)jz * g.ny + jy) * g.nx + jx;
    }
    const VofRec R = rec[up];
    if (R.p < 0.f) {
        // uniform upwind cell: phi_up u dt / h in FP64 (two products), so that a run of full or
        // empty cells gives F_{i+1/2} - F_{i-1/2} = phi (c_{i+1/2} - c_{i-1/2}) to FP64 rounding,
        // the same number the split update divides out, and phi stays in [0, 1] there
        const double cs = s == 0 ? g.c[0] : (s == 1 ? g.c[1] : g.c[2]);
        F[cell] = __ldg(&phi[up]) * (__ldg(&vel[cell]) * cs);
        return;
    }
    float v;
    {
        const int p = (int)R.p;
        const int o1 = p == 0 ? 1 : 0, o2 = p == 2 ? 1 : 2;
        // the swept interval along s, [0, 1] along the two other directions
        const float slo = c >= 0.f ? 1.f - c : 0.f, shi = c >= 0.f ? 1.f : -c;
        v = box_int(R, g.beta, p == s ? slo : 0.f, p == s ? shi : 1.f, o1 == s ? slo : 0.f, o1 == s ? shi : 1.f,
                    o2 == s ? slo : 0.f, o2 == s ? shi : 1.f);
    }
    F[cell] = f2d_bits(c >= 0.f ? v : -v);
}

// phi^p = (phi^s - (F_{i+1/2} - F_{i-1/2})) / (1 - dt/h (u_{i+1/2} - u_{i-1/2})).
__global__ void __launch_bounds__(512) k_vof_update(const double* __restrict__ phs, const double* __restrict__ F,
                                                    const double* __restrict__ vel, double* __restrict__ php,
                                                    VofGeo g, int s) {
    int ix, iy, iz;
    tile_cell(ix, iy, iz);
    const size_t cell = ((size_t)iz * g.ny + iy) * g.nx + ix;
    int jx = ix, jy = iy, jz = iz;
    if (s == 0) jx = ix == 0 ? g.nx - 1 : ix - 1;
    else if (s == 1) jy = iy == 0 ? g.ny - 1 : iy - 1;
    else jz = iz == 0 ? g.nz - 1 : iz - 1;
    const size_t lo = ((size_t)jz * g.ny + jy) * g.nx + jx;
    const double div = (s == 0 ? g.c[0] : (s == 1 ? g.c[1] : g.c[2])) * (vel[cell] - vel[lo]);
    php[cell] = (phs[cell] - (F[cell] - F[lo])) * rcp64(1.0 - div);
}

// phi^{n+1} = phi^z - sum_p dt/h_p phi^p (u_{i+1/2} - u_{i-1/2})_p.
__global__ void __launch_bounds__(512) k_vof_final(const double* __restrict__ st, const double* __restrict__ u,
                                                   const double* __restrict__ v, const double* __restrict__ w,
                                                   double* __restrict__ phi, VofGeo g) {
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    int ix, iy, iz;
    tile_cell(ix, iy, iz);
    const size_t cell = ((size_t)iz * g.ny + iy) * g.nx + ix;
    const size_t sx = ((size_t)iz * g.ny + iy) * g.nx + (ix == 0 ? g.nx - 1 : ix - 1);
    const size_t sy = ((size_t)iz * g.ny + (iy == 0 ? g.ny - 1 : iy - 1)) * g.nx + ix;
    const size_t sz = ((size_t)(iz == 0 ? g.nz - 1 : iz - 1) * g.ny + iy) * g.nx + ix;
    const double px = st[cell], py = st[N + cell], pz = st[2 * N + cell];
    double out = pz;
    out = out - g.c[0] * px * (u[cell] - u[sx]);
    out = out - g.c[1] * py * (v[cell] - v[sy]);
    out = out - g.c[2] * pz * (w[cell] - w[sz]);
    phi[cell] = out;
}

}  // namespace

// Plan-owned workspace of the VoF step: records (8 floats), face fluxes, the three stages.
static cudaError_t vof_workspace(flups_plan P) {
    if (P->vofbuf) return cudaSuccess;
    const size_t N = P->npts;
    const size_t bytes = N * sizeof(VofRec) + N * sizeof(double) + 3 * N * sizeof(double);
    void* b = nullptr;
    const cudaError_t e = cudaMalloc(&b, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return e; }
    P->vofbuf = b;
    return cudaSuccess;
}

extern "C" flups_status flups_vof_step(flups_plan P, double* phi, const double* u, const double* v,
                                       const double* w, double dt, double beta, double* stages) {
    NvtxRange nvtx_("flups_vof_step");
    if (!P || !phi || !u || !v || !w) return FLUPS_EINVAL;
    if (!(dt > 0.0) || !(beta > 0.0) || !std::isfinite(dt) || !std::isfinite(beta)) return FLUPS_EINVAL;
    if (P->bc != FLUPS_BC_PERIODIC || P->bcx != FLUPS_XY_PERIODIC || P->bcy != FLUPS_XY_PERIODIC)
        return FLUPS_EUNSUPPORTED;
    if (P->nx % VT || P->ny % VT || P->nz % VT) return FLUPS_EUNSUPPORTED;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != P->dev) cudaSetDevice(P->dev);
    cudaError_t e = vof_workspace(P);
    if (e != cudaSuccess) {
        if (dev != P->dev) cudaSetDevice(dev);
        flups_note_cuda_error(e);
        return FLUPS_ENOMEM;
    }
    const size_t N = P->npts;
    VofRec* rec = reinterpret_cast<VofRec*>(P->vofbuf);
    double* F = reinterpret_cast<double*>(rec + N);
    double* st = stages ? stages : F + N;
    VofGeo g;
    g.nx = P->nx; g.ny = P->ny; g.nz = P->nz;
    g.dt = dt;
    g.h[0] = P->dx; g.h[1] = P->dy; g.h[2] = P->dz0;
    for (int a = 0; a < 3; ++a) {
        g.c[a] = dt / g.h[a];
        g.cf[a] = (float)g.c[a];
    }
    g.beta = (float)beta;
    const double* vel[3] = {u, v, w};
    const dim3 rgrid(P->nx / VT, P->ny / VT, P->nz / VT);
    const int tb = VT * VT * VT;
    const double* src = phi;
    for (int s = 0; s < 3; ++s) {
        flups_prof_begin(P, FK_VOF_REC);
        k_vof_rec<<<rgrid, tb, 0, P->stream>>>(src, rec, g);
        flups_prof_end(P);
        flups_prof_begin(P, FK_VOF_FLUX);
        k_vof_flux<<<rgrid, tb, 0, P->stream>>>(src, rec, vel[s], F, g, s, &P->sc->vof_bad);
        flups_prof_end(P);
        flups_prof_begin(P, FK_VOF_UPDATE);
        k_vof_update<<<rgrid, tb, 0, P->stream>>>(src, F, vel[s], st + s * N, g, s);
        flups_prof_end(P);
        src = st + s * N;
    }
    flups_prof_begin(P, FK_VOF_UPDATE);
    k_vof_final<<<rgrid, tb, 0, P->stream>>>(st, u, v, w, phi, g);
    flups_prof_end(P);
    FLUPS_COUNT(P, 10);
    e = cudaGetLastError();
    if (dev != P->dev) cudaSetDevice(dev);
    if (e != cudaSuccess) {
        flups_note_cuda_error(e);
        return FLUPS_ECUDA;
    }
    return FLUPS_OK;
}
