// momentum.cu - the momentum predictor of one phase on a triply periodic MAC grid
// (Sec. 3.3, Eq. uss_predic), the step in front of the projection:
//
//   M^n  = -D(u^n u^n) + nu L u^n
//   u**  = u^n + dt (f1 M^n - f2 M^{n-1} + g),   f1 = 1 + dt/(2 dt_prev),  f2 = dt/(2 dt_prev)
//
// The convective flux is in divergence form built from two-point averages (u u at cell
// centres, u v, u w, v w on cell edges) and L is the 7-point Laplacian: central differences,
// as Sec. 3.3 states.  Constant density and viscosity, so the surface-tension term vanishes
// and the body force is the constant acceleration g.
//
// Tiling: a CTA covers RX x 8 columns (RX = min(32, nx)) and marches MOM_KC planes up z.
// u, v, w planes (tile plus a one-cell halo) and the own cells' M^{n-1} arrive by cp.async
// in a four-plane shared-memory ring two planes ahead of the computation (no register
// staging), are converted into a three-plane work ring, and each thread computes its column.
//
// Arithmetic.  GB300 issues binary64 at about 1/64 of the binary32 rate, and a binary64
// stencil of this size (~66 FP64 operations per cell) would run several times longer than
// its HBM traffic.  The default path therefore computes M in pairs of binary32 numbers on a
// fixed-point grid:
//   * a pre-pass finds E with max(|u|, |v|, |w|) < 2^E; every velocity is split into
//     A + a, A a multiple of q = 2^(E-20) (|A| <= 2^20 q) and a the binary32 remainder, so
//     every sum of up to twelve A's that the stencil forms is exact in binary32;
//   * each product of two such sums (|.| <= 2^42 q^2) is taken exactly with an FMA (Dekker's
//     product) and its high part rounded to a multiple of Q = 2^21 q^2, the remainder moving
//     to the low part, so the flux differences and their sums are exact too;
//   * the low parts (products with remainders, FMA errors, rounding remainders) are carried
//     in binary32, and the scalings by -1/(4h), nu/h^2, f1, f2, dt in pair arithmetic
//     (Knuth's TwoSum, Dekker's product).
// The error of M is then about 2^-38 max|u|^2 / h (binary64 gives ~2^-50), i.e. ~1e-12
// max|u| in u** at a CFL number of one.  The pair path needs dx = dy = dz and E inside a
// range that keeps every binary32 quantity normal; outside it the kernel runs the binary64
// path, which is also selectable (FLUPS_MOM_FP64) and handles any spacings.
//
// M state: M^n is stored for the next call as pairs (hi, lo) of binary32 (48 significant
// bits), [3][nz][ny][nx] float2; u** is binary64.
#include "flups_impl.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace {

constexpr int MOM_TY = 8;
constexpr int MOM_KC = 32;
constexpr int MOM_EMIN = -40;

struct Pf { float h, l; };

struct MomArgs {
    const double* u; const double* v; const double* w;
    double* us; double* vs; double* ws;
    float2* ms;                   // [3][n] M^{n-1} in, M^n out
    const unsigned int* hmax;     // high word of max(|u|, |v|, |w|) (pair path)
    int nx, ny, nz, kc, ab2, emin, emax;
    long long n;
    // binary64 path
    double idx4, idy4, idz4;      // -1/(4h)
    double nsx, nsy, nsz;         // nu/h^2
    double f1, mf2, dt, g[3];
    // pair path (dx = dy = dz = h)
    Pf sc, sl, F1, MF2, DT, G[3];
};

// ---------------------------------------------------------------- binary32 building blocks

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ Pf two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// x * c for pairs, to first order in the low parts: (t, lo), t = fl(x.h c.h) and its exact
// rounding error folded into lo (Dekker's product through an FMA).
__device__ __forceinline__ Pf mul_pc(Pf x, Pf c) {
    const float t = __fmul_rn(x.h, c.h);
    const float e = __fmaf_rn(x.h, c.h, -t);
    return {t, __fmaf_rn(x.h, c.l, __fmaf_rn(x.l, c.h, e))};
}

__device__ __forceinline__ Pf add_pp(Pf x, Pf y) {
    const Pf s = two_sum(x.h, y.h);
    return {s.h, s.l + x.l + y.l};
}

// x = h + l + r: h is x truncated to 24 significant bits, l the next 29 bits rounded to
// binary32, |r| <= 2^-47 |x|.  Integer operations and one integer-to-float conversion only
// (no binary64 instruction).  |x| < 2^-126 gives h = l = 0; requires |x| < 2^128.
__device__ __forceinline__ Pf split_d(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
    const unsigned int e = (hi >> 20) & 0x7FFu;
    const unsigned int sg = hi & 0x80000000u;
    unsigned int hb = sg | ((((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29));
    hb = e < 897u ? sg : hb;
    const float sc = e < 949u ? 0.f : __uint_as_float((e - 948u) << 23);   // 2^(e - 1075)
    const float l = __uint2float_rn(lo & 0x1FFFFFFFu) * sc;
    return {__uint_as_float(hb), __uint_as_float(__float_as_uint(l) ^ sg)};
}

// binary32 -> binary64 from the bit layouts (exact; zero and subnormals give a signed zero).
__device__ __forceinline__ double f2d_int(float x) {
    const unsigned int b = __float_as_uint(x);
    const unsigned int e = (b >> 23) & 0xFFu;
    const unsigned int sg = b & 0x80000000u;
    const unsigned int hi = e == 0u ? sg : (sg | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3));
    const unsigned int lo = e == 0u ? 0u : (b << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// (A, a): A = x.h rounded to a multiple of q (Kq = 1.5 * 2^23 q, |x.h| <= 2^22 q), a = the rest.
__device__ __forceinline__ float2 quant(Pf x, float Kq) {
    const float A = __fsub_rn(__fadd_rn(x.h, Kq), Kq);
    return make_float2(A, __fadd_rn(__fsub_rn(x.h, A), x.l));
}

// Product of two sums of quantised velocities, (X1 + X2)(Y1 + Y2): high part a multiple of
// Q (KQ = 1.5 * 2^23 Q), everything else in the low part.
__device__ __forceinline__ Pf prod2(float2 x1, float2 x2, float2 y1, float2 y2, float KQ) {
    const float S = __fadd_rn(x1.x, x2.x), s = x1.y + x2.y;   // S exact
    const float T = __fadd_rn(y1.x, y2.x), t = y1.y + y2.y;
    const float p = __fmul_rn(S, T);
    const float e = __fmaf_rn(S, T, -p);                      // exact
    const float c = __fmaf_rn(s, T + t, __fmaf_rn(S, t, e));
    const float pq = __fsub_rn(__fadd_rn(p, KQ), KQ);
    return {pq, c + __fsub_rn(p, pq)};                        // p - pq exact
}

__device__ __forceinline__ Pf sq2(float2 x1, float2 x2, float KQ) {
    const float S = __fadd_rn(x1.x, x2.x), s = x1.y + x2.y;
    const float p = __fmul_rn(S, S);
    const float e = __fmaf_rn(S, S, -p);
    const float c = __fmaf_rn(s, __fmaf_rn(2.f, S, s), e);
    const float pq = __fsub_rn(__fadd_rn(p, KQ), KQ);
    return {pq, c + __fsub_rn(p, pq)};
}

// Laplacian numerator sum of the six neighbours minus 6 x centre: exact high part.
__device__ __forceinline__ Pf lap6(float2 xm, float2 xp, float2 ym, float2 yp, float2 zm, float2 zp, float2 c0) {
    const float H = __fmaf_rn(-6.f, c0.x, __fadd_rn(__fadd_rn(__fadd_rn(xm.x, xp.x), __fadd_rn(ym.x, yp.x)),
                                                    __fadd_rn(zm.x, zp.x)));
    const float L = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y) - 6.f * c0.y;
    return {H, L};
}

// f1 M - f2 M^{n-1} + g, times dt, in pairs.
__device__ __forceinline__ Pf ab2_pair(Pf m, float2 mp, int ab2, Pf F1, Pf MF2, Pf G, Pf DT) {
    Pf acc = mul_pc(m, F1);
    if (ab2) acc = add_pp(acc, mul_pc(Pf{mp.x, mp.y}, MF2));
    acc = add_pp(acc, G);
    return mul_pc(acc, DT);
}

// ------------------------------------------------------------------------------- the march

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int RX> struct MomTile {
    static constexpr int TY = MOM_TY, RS = RX + 2, FS = (TY + 2) * RS, NT = RX * TY, NH = 2 * RS + 2 * TY;
    // raw ring: 4 planes of u, v, w (tile + halo, binary64) filled by cp.async two planes ahead;
    // work ring: 3 planes in the arithmetic's form; M ring: 3 planes of the own cells' M^{n-1}
    static constexpr int RAW = 4 * 3 * FS * 8, WORK = 3 * 3 * FS * 8, MST = 3 * 3 * NT * 8;
    static constexpr int BYTES = RAW + WORK + MST;
};

// Shared-memory pipeline per CTA (planes p = k0-1 .. k0+kc): raw slot (p - k0 + 1) % 4, work
// slot (p - k0 + 1) % 3, M slot (p - k0) % 3.  Iteration kk (plane k = k0 + kk): wait until
// the copies of plane k+1 (and M of plane k) have landed, convert plane k+1 into the work ring,
// issue the copies of plane k+3 (and M of plane k+2), compute plane k.
template <int RX, bool PAIR>
__device__ __forceinline__ void mom_march(const MomArgs& a, unsigned char* smem, int E) {
    using Tv = typename std::conditional<PAIR, float2, double>::type;
    using G = MomTile<RX>;
    constexpr int TY = G::TY, RS = G::RS, FS = G::FS, NT = G::NT, NH = G::NH;
    static_assert(NH <= NT, "one halo cell per thread");
    double* R = reinterpret_cast<double*>(smem);                       // [4][3][FS]
    Tv* T = reinterpret_cast<Tv*>(smem + G::RAW);                      // [3][3][FS]
    float2* Ms = reinterpret_cast<float2*>(smem + G::RAW + G::WORK);   // [3][3][NT]
    const int tid = threadIdx.x, tx = tid % RX, ty = tid / RX;
    const int i0 = blockIdx.x * RX, j0 = blockIdx.y * TY, k0 = blockIdx.z * a.kc;
    const int c = (ty + 1) * RS + tx + 1;
    int hl = 0, hg = 0;
    if (tid < NH) {
        int lx, ly;
        if (tid < RS) { ly = 0; lx = tid; }
        else if (tid < 2 * RS) { ly = TY + 1; lx = tid - RS; }
        else if (tid < 2 * RS + TY) { ly = tid - 2 * RS + 1; lx = 0; }
        else { ly = tid - 2 * RS - TY + 1; lx = RS - 1; }
        hl = ly * RS + lx;
        hg = ((j0 + ly - 1) & (a.ny - 1)) * a.nx + ((i0 + lx - 1) & (a.nx - 1));
    }
    const int og = (j0 + ty) * a.nx + i0 + tx;
    const long long plane = (long long)a.nx * a.ny;
    float Kq = 0.f, KQ = 0.f;
    if constexpr (PAIR) {
        Kq = __uint_as_float(((unsigned int)(E + 3 + 127) << 23) | 0x400000u);       // 1.5 * 2^23 q
        KQ = __uint_as_float(((unsigned int)(2 * E + 4 + 127) << 23) | 0x400000u);   // 1.5 * 2^23 Q
    }
    auto issue_raw = [&](int p) {                  // plane p (unwrapped) into its raw slot
        const long long base = (long long)(p & (a.nz - 1)) * plane;
        double* dst = R + ((p - k0 + 1) & 3) * 3 * FS;
        cp_async8(dst + c, a.u + base + og);
        cp_async8(dst + FS + c, a.v + base + og);
        cp_async8(dst + 2 * FS + c, a.w + base + og);
        if (tid < NH) {
            cp_async8(dst + hl, a.u + base + hg);
            cp_async8(dst + FS + hl, a.v + base + hg);
            cp_async8(dst + 2 * FS + hl, a.w + base + hg);
        }
    };
    auto issue_m = [&](int p) {                    // M^{n-1} of the own cells of plane p
        if (!a.ab2) return;
        float2* dst = Ms + ((p - k0) % 3) * 3 * NT + tid;
        const long long o = (long long)p * plane + og;
#pragma unroll
        for (int f = 0; f < 3; ++f) cp_async8(dst + f * NT, a.ms + f * a.n + o);
    };
    auto cvt = [&](double x) -> Tv {
        if constexpr (PAIR) return quant(split_d(x), Kq);
        else return x;
    };
    auto convert = [&](int p) {                    // raw plane p -> work ring
        const double* src = R + ((p - k0 + 1) & 3) * 3 * FS;
        Tv* dst = T + ((p - k0 + 1) % 3) * 3 * FS;
#pragma unroll
        for (int f = 0; f < 3; ++f) dst[f * FS + c] = cvt(src[f * FS + c]);
        if (tid < NH) {
#pragma unroll
            for (int f = 0; f < 3; ++f) dst[f * FS + hl] = cvt(src[f * FS + hl]);
        }
    };
    // products on the k-1/2 faces, carried from the previous plane's k+1/2 ones
    Pf c_uw = {0.f, 0.f}, c_vw = {0.f, 0.f}, c_ww = {0.f, 0.f};
    double d_uw = 0.0, d_vw = 0.0, d_ww = 0.0;
    issue_raw(k0 - 1); cp_commit();
    issue_raw(k0); cp_commit();
    issue_raw(k0 + 1); issue_m(k0); cp_commit();
    issue_raw(k0 + 2); issue_m(k0 + 1); cp_commit();
    cp_wait<2>();
    __syncthreads();
    convert(k0 - 1);
    convert(k0);

    for (int kk = 0; kk < a.kc; ++kk) {
        const int k = k0 + kk;
        cp_wait<1>();                              // raw plane k+1 and M of plane k have landed
        __syncthreads();                           // ... for every thread; plane k-2's work slot is free
        convert(k + 1);
        if (kk + 3 <= a.kc) { issue_raw(k + 3); issue_m(k + 2); }
        cp_commit();
        __syncthreads();
        const long long o = (long long)k * plane + og;
        const Tv* Xm = T + (kk % 3) * 3 * FS + c;
        const Tv* X0 = T + ((kk + 1) % 3) * 3 * FS + c;
        const Tv* Xp = T + ((kk + 2) % 3) * 3 * FS + c;
        const double* own = R + ((kk + 1) & 3) * 3 * FS + c;
        const float2* mprev = Ms + (kk % 3) * 3 * NT + tid;
        // u: field 0, v: field 1, w: field 2
        const Tv U0 = X0[0], Uxm = X0[-1], Uxp = X0[1], Uym = X0[-RS], Uyp = X0[RS], Uzm = Xm[0], Uzp = Xp[0];
        const Tv Uxm_yp = X0[RS - 1], Uxm_zp = Xp[-1];
        const Tv V0 = X0[FS], Vxm = X0[FS - 1], Vxp = X0[FS + 1], Vym = X0[FS - RS], Vyp = X0[FS + RS];
        const Tv Vzm = Xm[FS], Vzp = Xp[FS], Vxp_ym = X0[FS + 1 - RS], Vym_zp = Xp[FS - RS];
        const Tv W0 = X0[2 * FS], Wxm = X0[2 * FS - 1], Wxp = X0[2 * FS + 1], Wym = X0[2 * FS - RS];
        const Tv Wyp = X0[2 * FS + RS], Wzm = Xm[2 * FS], Wzp = Xp[2 * FS], Wxp_zm = Xm[2 * FS + 1];
        const Tv Wyp_zm = Xm[2 * FS + RS];
        float2 mp[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (a.ab2) {
#pragma unroll
            for (int f = 0; f < 3; ++f) mp[f] = mprev[f * NT];
        }
        double res[3];
        float2 mout[3];
        if constexpr (PAIR) {
            // fluxes (products of two-point sums; the 1/4 of the averages is in sc)
            const Pf uu_i = sq2(Uxm, U0, KQ), uu_ip = sq2(U0, Uxp, KQ);
            const Pf vv_j = sq2(Vym, V0, KQ), vv_jp = sq2(V0, Vyp, KQ);
            if (kk == 0) {
                c_ww = sq2(Wzm, W0, KQ);
                c_uw = prod2(Uzm, U0, Wzm, Wxp_zm, KQ);            // (i+1/2, k-1/2)
                c_vw = prod2(Vzm, V0, Wzm, Wyp_zm, KQ);            // (j+1/2, k-1/2)
            }
            const Pf ww_k = c_ww, ww_kp = sq2(W0, Wzp, KQ);
            const Pf uv_pp = prod2(U0, Uyp, V0, Vxp, KQ);          // edge (i+1/2, j+1/2)
            const Pf uv_pm = prod2(Uym, U0, Vym, Vxp_ym, KQ);      // (i+1/2, j-1/2)
            const Pf uv_mp = prod2(Uxm, Uxm_yp, Vxm, V0, KQ);      // (i-1/2, j+1/2)
            const Pf uw_pp = prod2(U0, Uzp, W0, Wxp, KQ);          // (i+1/2, k+1/2)
            const Pf uw_pm = c_uw;
            const Pf uw_mp = prod2(Uxm, Uxm_zp, Wxm, W0, KQ);      // (i-1/2, k+1/2)
            const Pf vw_pp = prod2(V0, Vzp, W0, Wyp, KQ);          // (j+1/2, k+1/2)
            const Pf vw_pm = c_vw;
            const Pf vw_mp = prod2(Vym, Vym_zp, Wym, W0, KQ);      // (j-1/2, k+1/2)
            c_ww = ww_kp; c_uw = uw_pp; c_vw = vw_pp;
            auto div3 = [](Pf a1, Pf b1, Pf a2, Pf b2, Pf a3, Pf b3) -> Pf {
                const float H = __fadd_rn(__fadd_rn(__fsub_rn(a1.h, b1.h), __fsub_rn(a2.h, b2.h)), __fsub_rn(a3.h, b3.h));
                return {H, ((a1.l - b1.l) + (a2.l - b2.l)) + (a3.l - b3.l)};
            };
            const Pf cu = div3(uu_ip, uu_i, uv_pp, uv_pm, uw_pp, uw_pm);
            const Pf cv = div3(uv_pp, uv_mp, vv_jp, vv_j, vw_pp, vw_pm);
            const Pf cw = div3(uw_pp, uw_mp, vw_pp, vw_mp, ww_kp, ww_k);
            const Pf lu = lap6(Uxm, Uxp, Uym, Uyp, Uzm, Uzp, U0);
            const Pf lv = lap6(Vxm, Vxp, Vym, Vyp, Vzm, Vzp, V0);
            const Pf lw = lap6(Wxm, Wxp, Wym, Wyp, Wzm, Wzp, W0);
            const Pf M[3] = {add_pp(mul_pc(cu, a.sc), mul_pc(lu, a.sl)), add_pp(mul_pc(cv, a.sc), mul_pc(lv, a.sl)),
                             add_pp(mul_pc(cw, a.sc), mul_pc(lw, a.sl))};
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const Pf d = ab2_pair(M[f], mp[f], a.ab2, a.F1, a.MF2, a.G[f], a.DT);
                res[f] = (own[f * FS] + f2d_int(d.h)) + f2d_int(d.l);
                mout[f] = make_float2(M[f].h, M[f].l);
            }
        } else {
            const double uu_i = (Uxm + U0) * (Uxm + U0), uu_ip = (U0 + Uxp) * (U0 + Uxp);
            const double vv_j = (Vym + V0) * (Vym + V0), vv_jp = (V0 + Vyp) * (V0 + Vyp);
            if (kk == 0) {
                d_ww = (Wzm + W0) * (Wzm + W0);
                d_uw = (Uzm + U0) * (Wzm + Wxp_zm);
                d_vw = (Vzm + V0) * (Wzm + Wyp_zm);
            }
            const double ww_k = d_ww, ww_kp = (W0 + Wzp) * (W0 + Wzp);
            const double uv_pp = (U0 + Uyp) * (V0 + Vxp), uv_pm = (Uym + U0) * (Vym + Vxp_ym);
            const double uv_mp = (Uxm + Uxm_yp) * (Vxm + V0);
            const double uw_pp = (U0 + Uzp) * (W0 + Wxp), uw_pm = d_uw;
            const double uw_mp = (Uxm + Uxm_zp) * (Wxm + W0);
            const double vw_pp = (V0 + Vzp) * (W0 + Wyp), vw_pm = d_vw;
            const double vw_mp = (Vym + Vym_zp) * (Wym + W0);
            d_ww = ww_kp; d_uw = uw_pp; d_vw = vw_pp;
            const double M[3] = {
                (uu_ip - uu_i) * a.idx4 + (uv_pp - uv_pm) * a.idy4 + (uw_pp - uw_pm) * a.idz4 +
                    (Uxm + Uxp - 2.0 * U0) * a.nsx + (Uym + Uyp - 2.0 * U0) * a.nsy + (Uzm + Uzp - 2.0 * U0) * a.nsz,
                (uv_pp - uv_mp) * a.idx4 + (vv_jp - vv_j) * a.idy4 + (vw_pp - vw_pm) * a.idz4 +
                    (Vxm + Vxp - 2.0 * V0) * a.nsx + (Vym + Vyp - 2.0 * V0) * a.nsy + (Vzm + Vzp - 2.0 * V0) * a.nsz,
                (uw_pp - uw_mp) * a.idx4 + (vw_pp - vw_mp) * a.idy4 + (ww_kp - ww_k) * a.idz4 +
                    (Wxm + Wxp - 2.0 * W0) * a.nsx + (Wym + Wyp - 2.0 * W0) * a.nsy + (Wzm + Wzp - 2.0 * W0) * a.nsz};
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                double acc = a.f1 * M[f];
                if (a.ab2) acc += a.mf2 * ((double)mp[f].x + (double)mp[f].y);
                res[f] = own[f * FS] + a.dt * (acc + a.g[f]);
                const float h = __double2float_rn(M[f]);
                mout[f] = make_float2(h, __double2float_rn(M[f] - (double)h));
            }
        }
        a.us[o] = res[0]; a.vs[o] = res[1]; a.ws[o] = res[2];
#pragma unroll
        for (int f = 0; f < 3; ++f) a.ms[f * a.n + o] = mout[f];
    }
    cp_wait<0>();
}

template <int RX, bool PAIR>
__global__ void __launch_bounds__(RX * MOM_TY, RX == 32 ? 3 : 4) k_momentum(MomArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (PAIR) {
        const unsigned int hm = *a.hmax;
        const int E = hm == 0u ? 0 : (int)(hm >> 20) - 1022;
        if (E >= a.emin && E <= a.emax) {
            mom_march<RX, true>(a, smem, E);
            return;
        }
    }
    mom_march<RX, false>(a, smem, 0);
}

// High word (sign cleared) of max over u, v, w: its exponent field bounds max|.|.
__global__ void __launch_bounds__(256) k_mom_umax(const double* __restrict__ u, const double* __restrict__ v,
                                                  const double* __restrict__ w, long long n, unsigned int* hmax) {
    unsigned int m = 0u;
    const long long n2 = n >> 1;
    const uint4* U = reinterpret_cast<const uint4*>(u);
    const uint4* V = reinterpret_cast<const uint4*>(v);
    const uint4* W = reinterpret_cast<const uint4*>(w);
    for (long long t = blockIdx.x * 256LL + threadIdx.x; t < n2; t += (long long)gridDim.x * 256) {
        const uint4 x = __ldg(U + t), y = __ldg(V + t), z = __ldg(W + t);
        m = max(m, max(x.y & 0x7FFFFFFFu, x.w & 0x7FFFFFFFu));
        m = max(m, max(max(y.y & 0x7FFFFFFFu, y.w & 0x7FFFFFFFu), max(z.y & 0x7FFFFFFFu, z.w & 0x7FFFFFFFu)));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    __shared__ unsigned int wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) m = max(m, wm[q]);
        atomicMax(hmax, m);
    }
}

Pf pair_of(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

bool overlaps(const void* a, const void* b, size_t bytes_a, size_t bytes_b) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + bytes_b && pb < pa + bytes_a;
}

template <int RX>
cudaError_t launch_mom(flups_plan P, const MomArgs& a, bool pair) {
    const dim3 grid(P->nx / RX, P->ny / MOM_TY, P->nz / a.kc);
    constexpr int bytes = MomTile<RX>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_momentum<RX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_momentum<RX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    if (pair) k_momentum<RX, true><<<grid, RX * MOM_TY, bytes, P->stream>>>(a);
    else k_momentum<RX, false><<<grid, RX * MOM_TY, bytes, P->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

extern "C" flups_status flups_momentum_predict(flups_plan P, const double* u, const double* v, const double* w,
                                               double* us, double* vs, double* ws, void* m_state, double nu,
                                               double gx, double gy, double gz, double dt, double dt_prev,
                                               int arith) {
    NvtxRange nvtx_("flups_momentum_predict");
    if (!P || !u || !v || !w || !us || !vs || !ws || !m_state) return FLUPS_EINVAL;
    const void* ptrs[7] = {u, v, w, us, vs, ws, m_state};
    for (const void* p : ptrs)
        if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return FLUPS_EINVAL;
    const size_t fb = P->npts * sizeof(double);
    const size_t sizes[7] = {fb, fb, fb, fb, fb, fb, 3 * P->npts * sizeof(float2)};
    for (int x = 3; x < 7; ++x)            // outputs may not overlap each other or any input
        for (int y = 0; y < 7; ++y)
            if (x != y && overlaps(ptrs[x], ptrs[y], sizes[x], sizes[y])) return FLUPS_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(dt_prev) || !(nu >= 0.0) || !std::isfinite(nu) ||
        !std::isfinite(gx) || !std::isfinite(gy) || !std::isfinite(gz))
        return FLUPS_EINVAL;
    if (arith != FLUPS_MOM_PAIR && arith != FLUPS_MOM_FP64) return FLUPS_EINVAL;
    if (P->bc != FLUPS_BC_PERIODIC || P->bcx != FLUPS_XY_PERIODIC || P->bcy != FLUPS_XY_PERIODIC)
        return FLUPS_EUNSUPPORTED;
    const double dz = P->dz0;             // periodic z: uniform spacing
    const double h = P->dx;
    if (arith == FLUPS_MOM_PAIR && !P->uniform_h) return FLUPS_EUNSUPPORTED;
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != P->dev) cudaSetDevice(P->dev);
    else prev = -1;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};

    MomArgs a;
    a.u = u; a.v = v; a.w = w; a.us = us; a.vs = vs; a.ws = ws;
    a.ms = static_cast<float2*>(m_state);
    a.hmax = &P->sc->mom_hmax;
    a.nx = P->nx; a.ny = P->ny; a.nz = P->nz;
    a.kc = P->nz < MOM_KC ? P->nz : MOM_KC;
    a.n = (long long)P->npts;
    a.ab2 = dt_prev > 0.0;
    const double r = a.ab2 ? dt / dt_prev : 0.0;
    a.f1 = 1.0 + 0.5 * r;
    a.mf2 = -0.5 * r;
    a.dt = dt;
    a.g[0] = gx; a.g[1] = gy; a.g[2] = gz;
    a.idx4 = -0.25 / P->dx; a.idy4 = -0.25 / P->dy; a.idz4 = -0.25 / dz;
    a.nsx = nu / (P->dx * P->dx); a.nsy = nu / (P->dy * P->dy); a.nsz = nu / (dz * dz);
    a.sc = pair_of(-0.25 / h);
    a.sl = pair_of(nu / (h * h));
    a.F1 = pair_of(a.f1); a.MF2 = pair_of(a.mf2); a.DT = pair_of(dt);
    for (int f = 0; f < 3; ++f) a.G[f] = pair_of(a.g[f]);
    // E range of the pair path: q = 2^(E-20) and Q = 2^(2E-19) normal, and the scaled flux
    // (<= 6 * 2^(2E) / h) and Laplacian (<= 12 * 2^E nu / h^2) terms below 2^126.
    a.emin = MOM_EMIN;
    int emax = 60;
    emax = std::min(emax, (int)std::floor((126.0 - std::log2(6.0 / h)) / 2.0) - 1);
    if (nu > 0.0) emax = std::min(emax, (int)std::floor(126.0 - std::log2(12.0 * nu / (h * h))) - 1);
    a.emax = emax;

    cudaStream_t s = P->stream;
    cudaError_t e = cudaSuccess;
    const bool pair = arith == FLUPS_MOM_PAIR;
    if (pair) {
        flups_prof_begin(P, FK_MOM_UMAX);
        e = cudaMemsetAsync(&P->sc->mom_hmax, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) {
            const long long n2 = a.n / 2;
            const int nb = (int)std::min<long long>((n2 + 255) / 256, 152LL * 8);
            k_mom_umax<<<nb, 256, 0, s>>>(u, v, w, a.n, &P->sc->mom_hmax);
            FLUPS_COUNT(P, 1);
            e = cudaGetLastError();
        }
        flups_prof_end(P);
    }
    if (e == cudaSuccess) {
        flups_prof_begin(P, FK_MOMENTUM);
        e = P->nx >= 32 ? launch_mom<32>(P, a, pair) : (P->nx == 16 ? launch_mom<16>(P, a, pair) : launch_mom<8>(P, a, pair));
        FLUPS_COUNT(P, 1);
        flups_prof_end(P);
    }
    if (e != cudaSuccess) {
        flups_note_cuda_error(e);
        return FLUPS_ECUDA;
    }
    return FLUPS_OK;
}
