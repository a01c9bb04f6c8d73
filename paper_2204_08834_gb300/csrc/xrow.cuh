// xrow.cuh - the register four-step transform of x rows (FluTAS Sec. 3.3.1, the transform
// along x): tile shape of the row kernels and the forward transform with the real-to-complex
// split from registers to the spectrum, shared by the row kernels and the defect pass.
//
// A row of nx reals is the complex sequence z[n] = x[2n] + i x[2n+1] of length M = N1 N2.
// Thread (c, t) of a tile of rows holds z[N2 n1 + t], n1 < N1, of row c.  The forward transform
// takes the N1-point DFT in registers, multiplies by W_M^(t k1), exchanges once through shared
// memory and takes the N2-point DFTs, so that the thread holds Z[k1 + N1 k2] for k1 = t + N2 q
// (q < N1/N2), k2 < N2.  The split
//   X_k = A_k + W_nx^k B_k,  A_k = (Z_k + conj Z_{M-k})/2,  B_k = (Z_k - conj Z_{M-k})/(2i)
// (k = 0..M-1, and X_M = A_0 - B_0) needs Z_{M-k}, which sits in lane N2 - t of the same row
// (lane 0 holds its own): one shuffle per value.  W_nx^k for k > M/2 is -conj(W_nx^(M-k)).
#pragma once
#include "blocksum.cuh"
#include "flups_impl.cuh"
#include "fp_bits.cuh"
#include "regfft.cuh"

namespace {

constexpr int XROW_THREADS = 256;

template <int N1, int N2>
struct XRow {
    static_assert(N1 >= N2 && N1 % N2 == 0 && N2 >= 8 && N2 <= 32, "row split");
    static constexpr int M = N1 * N2, Q = N1 / N2;
    static constexpr int B = XROW_THREADS / N2;   // rows per CTA
    // row pitch of the exchange area (complex values): room for N1 (N2 + 1) entries and for
    // the M + 1 spectrum values of the inverse's pairing step; congruent to 8 (mod 16) when
    // N2 = 8, so that the four rows a warp covers fall on distinct banks, else to 0.
    static constexpr int XP = ((N1 * (N2 + 1) + 15) / 16) * 16 + (N2 == 8 ? 8 : 0);
    static constexpr size_t SMEM = (size_t)B * XP * sizeof(float2);
};

// W_nx^k for 0 <= k < M from the table of W_nx^j, j <= M/2.
template <int M>
__device__ __forceinline__ float2 wsplit(const float2* __restrict__ twr, int k) {
    if (k <= M / 2) return __ldg(&twr[k]);
    const float2 w = __ldg(&twr[M - k]);
    return make_float2(-w.x, w.y);
}

// The forward transform of one row held as z[N2 n1 + t] in v (thread (c, t)), through the
// row's exchange area ex + c XP, and the split into the half spectrum row out (M + 1 values;
// stored when live).  Every thread of the CTA calls it (it holds a barrier); threads with
// active = false (whole warps) only take part in the barrier.
template <int N1, int N2>
__device__ __forceinline__ void xrow4_fwd_tail(float2 (&v)[N1], float2* __restrict__ ex, int c, int t, bool active,
                                               bool live, const float2* __restrict__ tw,
                                               const float2* __restrict__ twr, float2* __restrict__ out) {
    using X = XRow<N1, N2>;
    constexpr int M = X::M, Q = X::Q, XP = X::XP;
    float2* e = ex + c * XP;
    if (active) {
        RegDft<N1, false>::run(v);
        sfor<N1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            float2 a = v[k1];
            if (k1 > 0) a = tmul<false>(a, __ldg(&tw[(t * k1) & (M - 1)]));
            e[k1 * (N2 + 1) + t] = a;
        });
    }
    __syncthreads();
    if (!active) return;
    float2 w[Q][N2];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) w[q][n2] = e[(t + N2 * q) * (N2 + 1) + n2];
        RegDft<N2, false>::run(w[q]);
    }
    // the split, with Z_{M-k} from lane N2 - t (register (Q-1-q, N2-1-k2) there)
    const int plane = ((threadIdx.x & 31) & ~(N2 - 1)) | ((N2 - t) & (N2 - 1));
    sfor<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        sfor<N2>([&](auto k2c) {
            constexpr int k2 = decltype(k2c)::value;
            const float2 zk = w[q][k2];
            float2 zm;
            zm.x = __shfl_sync(0xffffffffu, w[Q - 1 - q][N2 - 1 - k2].x, plane);
            zm.y = __shfl_sync(0xffffffffu, w[Q - 1 - q][N2 - 1 - k2].y, plane);
            if (t == 0) zm = q == 0 ? w[0][(N2 - k2) % N2] : w[(Q - q) % Q][N2 - 1 - k2];
            const int k = t + N2 * q + N1 * k2;
            const float ax = (zk.x + zm.x) * 0.5f, ay = (zk.y - zm.y) * 0.5f;
            const float bxx = (zk.y + zm.y) * 0.5f, byy = (zm.x - zk.x) * 0.5f;
            const float2 wt = wsplit<M>(twr, k);
            const float tx = wt.x * bxx - wt.y * byy, ty = wt.x * byy + wt.y * bxx;
            if (live) {
                out[k] = make_float2(ax + tx, ay + ty);
                if (k == 0) out[M] = make_float2(ax - tx, ty - ay);
            }
        });
    });
}

// x = xh + xl for a binary64 x, by integer operations: xh = x with the low 29 significand bits
// cleared (exactly a binary32 number), xl = those 29 bits, rounded to binary32 (relative error
// 2^-24 of xl, so 2^-48 of x).  For |x| below 2^-126 both are 0 (the value is dropped); for
// |x| at or above 2^128, infinities and NaNs, xh is x rounded to binary32 (infinite or NaN).
__device__ __forceinline__ void split_d(double x, float& xh, float& xl) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FFu);
    const unsigned sgn = hi & 0x80000000u;
    if ((unsigned)(e - 897) <= 253u) {
        xh = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
        const int es = e - 948;             // the binary32 exponent field of 2^(e - 1075)
        const float sc = es >= 1 ? __uint_as_float((unsigned)es << 23) : 0.f;
        xl = __uint_as_float(__float_as_uint(__uint2float_rn(lo & 0x1FFFFFFFu) * sc) | sgn);
    } else {
        xh = e < 897 ? 0.f : d2f_bits(x);
        xl = 0.f;
    }
}

// (sh, sl) += a with an exact two-sum of sh and a (sl collects the rounding error).
__device__ __forceinline__ void two_sum_acc(float& sh, float& sl, float a) {
    const float s = sh + a, bb = s - sh;
    sl += (sh - (s - bb)) + (a - bb);
    sh = s;
}

// Forward: f (nx reals per row) -> the half spectrum S (M + 1 values per row, pitch ldS).
// STATS: also the partial sums sum_k dzf_k sum_ij f, sum f^2 and sum f of each CTA into part:
// a thread's row sum of f as a pair of binary32 numbers (f split into xh + xl, xh added by exact
// two-sums), so no FP64 instruction runs per point; sums of f^2 and f in FP32 per thread; all
// three in FP64 across threads.
template <int N1, int N2, bool STATS>
__device__ __forceinline__ void xrow4_fwd_body(int bx, const double* __restrict__ f, float2* __restrict__ S,
                                               const Geo& g, const float2* __restrict__ tw,
                                               const float2* __restrict__ twr, int nrows,
                                               double* __restrict__ part) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    using X = XRow<N1, N2>;
    extern __shared__ __align__(16) float2 ex[];
    const int tid = threadIdx.x, c = tid / N2, t = tid % N2;
    const int row = bx * X::B + c;
    const bool live = row < nrows;
    const double2* src = reinterpret_cast<const double2*>(f + (size_t)(live ? row : 0) * g.nx) + t;
    float2 v[N1];
    float sh = 0.f, sl = 0.f, acc2 = 0.f, acc1 = 0.f;
    // f in chunks of up to 16 loads (the row sums of a chunk are formed before the next loads)
    constexpr int CH = N1 < 16 ? N1 : 16;
#pragma unroll
    for (int h = 0; h < N1; h += CH) {
        double2 fv[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) fv[i] = live ? __ldg(src + N2 * (h + i)) : make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            v[h + i] = make_float2(d2f_bits(fv[i].x), d2f_bits(fv[i].y));
            if (STATS) {
                float h0, l0, h1, l1;
                split_d(fv[i].x, h0, l0);
                split_d(fv[i].y, h1, l1);
                two_sum_acc(sh, sl, h0);
                two_sum_acc(sh, sl, h1);
                sl += l0 + l1;
                acc2 = fmaf(v[h + i].x, v[h + i].x, fmaf(v[h + i].y, v[h + i].y, acc2));
                acc1 += v[h + i].x + v[h + i].y;
            }
        }
    }
    xrow4_fwd_tail<N1, N2>(v, ex, c, t, true, live, tw, twr, S + (size_t)(live ? row : 0) * g.ldS);
    if (STATS) {
        const double wz = live ? __ldg(g.dzf + row / g.ny) : 0.0;
        block_sum_abc<true, true, true>((f2d_bits(sh) + f2d_bits(sl)) * wz, acc2, acc1, part, bx);
    }
}


// The inverse forms Z_k = A_k + i conj(W_nx^k) D_k, A_k = (X_k + conj X_{M-k})/2,
// D_k = (X_k - conj X_{M-k})/2, with X_0 and X_M taken real, through shared memory (the partner
// of X_0 is X_M, not a lane's value), then runs the four steps backwards and ends in the
// layout the forward loads from.
// Inverse: S -> p (ACC = 0: p = x; ACC = 1: p += x, in FP64).  MEAN (with ACC = 0): the
// partial sums of dzf * p (the values are binary32 numbers: summed per thread in pairs of
// binary32 with exact two-sums, then in FP64); SUBM (with ACC = 1): x - <p_0> is added.  The
// largest binary64 exponent written goes to sc->pexp (the scale of the next defect).
// F32: the iterate is held in binary32 in p32 (rows of nx values, as p): with ACC = 0 x is
// stored there instead of in p (the values are binary32 numbers: nothing is lost), with ACC = 1
// the old iterate is read from there and the sum goes to p.
template <int N1, int N2, int ACC, bool MEAN, bool SUBM, bool F32>
__device__ __forceinline__ void xrow4_inv_body(int bx, const float2* __restrict__ S, double* __restrict__ p,
                                               float* __restrict__ p32, const Geo& g, const float2* __restrict__ tw,
                                               const float2* __restrict__ twr, int nrows,
                                               DevScalars* __restrict__ sc, double* __restrict__ part) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    using X = XRow<N1, N2>;
    constexpr int M = X::M, Q = X::Q, XP = X::XP;
    extern __shared__ __align__(16) float2 ex[];
    const int tid = threadIdx.x, c = tid / N2, t = tid % N2;
    const int row = bx * X::B + c;
    const bool live = row < nrows;
    const float2* in = S + (size_t)(live ? row : 0) * g.ldS;
    float2* e = ex + c * XP;
    float2 w[Q][N2];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int k = t + N2 * q + N1 * k2;
            w[q][k2] = live ? in[k] : make_float2(0.f, 0.f);
            e[k] = w[q][k2];
        }
    if (t == 0) e[M] = live ? in[M] : make_float2(0.f, 0.f);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int k = t + N2 * q + N1 * k2;
            float2 xk = w[q][k2], xm = e[M - k];
            if (k == 0) { xk.y = 0.f; xm.y = 0.f; }
            const float ax = (xk.x + xm.x) * 0.5f, ay = (xk.y - xm.y) * 0.5f;
            const float dx = (xk.x - xm.x) * 0.5f, dy = (xk.y + xm.y) * 0.5f;
            const float2 wt = wsplit<M>(twr, k);
            const float bxx = dx * wt.x + dy * wt.y, byy = dy * wt.x - dx * wt.y;
            w[q][k2] = make_float2(ax - byy, ay + bxx);
        }
#pragma unroll
    for (int q = 0; q < Q; ++q) RegDft<N2, true>::run(w[q]);
    __syncthreads();                        // every pairing read is done: the area takes the exchange
    sfor<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const int k1 = t + N2 * q;
        sfor<N2>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            float2 a = w[q][n2];
            if (n2 > 0) a = tmul<true>(a, __ldg(&tw[(n2 * k1) & (M - 1)]));
            e[k1 * (N2 + 1) + n2] = a;
        });
    });
    double2* dst = reinterpret_cast<double2*>(p + (size_t)(live ? row : 0) * g.nx) + t;
    float2* d32 = reinterpret_cast<float2*>(p32 + (size_t)(live ? row : 0) * g.nx) + t;
    auto old_p = [&](int n1) {
        if (F32) {
            const float2 o = live ? d32[N2 * n1] : make_float2(0.f, 0.f);
            return make_double2(f2d_bits(o.x), f2d_bits(o.y));
        }
        return live ? dst[N2 * n1] : make_double2(0.0, 0.0);
    };
    // p += x: the old p is loaded before the last exchange and DFT (where the registers allow)
    constexpr bool PRE = ACC && N1 <= 16;
    double2 pold[PRE ? N1 : 1];
    if (PRE) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) pold[PRE ? n1 : 0] = old_p(n1);
    }
    __syncthreads();
    float2 v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = e[k1 * (N2 + 1) + t];
    RegDft<N1, true>::run(v);
    float msub = 0.f;
    if (SUBM) msub = (float)sc->mean_p;
    int emax = 0;
    unsigned int fmax_bits = 0u;            // F32 && !ACC: the largest binary32 exponent field (in place)
    float sh = 0.f, sl = 0.f;               // the binary32 pair sum of MEAN
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
        float2 z = v[n1];
        if (SUBM) { z.x -= msub; z.y -= msub; }
        if constexpr (F32 && !ACC) {
            // binary32 store; the exponent is read from the binary32 bits (mapped to the binary64
            // field after the loop), with no conversion of the value
            if (MEAN) {
                two_sum_acc(sh, sl, z.x);
                two_sum_acc(sh, sl, z.y);
            }
            if (live) d32[N2 * n1] = z;
            fmax_bits = max(fmax_bits, max(__float_as_uint(z.x) & 0x7F800000u, __float_as_uint(z.y) & 0x7F800000u));
        } else {
            double2 o;
            if (ACC) {
                if (PRE) o = pold[PRE ? n1 : 0];
                else o = old_p(n1);
                o.x += f2d_bits(z.x);
                o.y += f2d_bits(z.y);
            } else {
                o = make_double2(f2d_bits(z.x), f2d_bits(z.y));
                if (MEAN) {
                    two_sum_acc(sh, sl, z.x);
                    two_sum_acc(sh, sl, z.y);
                }
            }
            if (live) dst[N2 * n1] = o;
            const int ex_ = (int)((__double_as_longlong(o.x) >> 52) & 0x7FF);
            const int ey_ = (int)((__double_as_longlong(o.y) >> 52) & 0x7FF);
            emax = max(emax, max(ex_, ey_));
        }
    }
    if constexpr (F32 && !ACC) {
        // the binary64 field of (double)x: 0 for zero and binary32 subnormals (f2d_bits flushes
        // them), e + 896 for normal numbers, 2047 for infinities and NaNs
        const int e32 = (int)(fmax_bits >> 23);
        emax = e32 == 0 ? 0 : (e32 == 255 ? 2047 : e32 + 896);
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((tid & 31) == 0) atomicMax(&sc->pexp, emax);
    if (MEAN) {
        const double wz = live ? __ldg(g.dzf + row / g.ny) : 0.0;
        block_sum_abc<true, false, false>((f2d_bits(sh) + f2d_bits(sl)) * wz, 0.f, 0.f, part, bx);
    }
}


}  // namespace
