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
#include "flups_impl.cuh"
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

}  // namespace
