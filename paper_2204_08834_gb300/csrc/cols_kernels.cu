// cols_kernels.cu - FP32 column transforms of the eigen-expansion solver held in registers
// (FluTAS Sec. 3.3.1, steps 3, 5 and 7: the transform along y, and with a periodic z the
// transform along z, the division by the eigenvalues and the inverse z transform).
//
// A column of length N = N1 N2 (powers of two, N1 >= N2) is transformed in four steps:
//   X[k1 + N1 k2] = sum_n2 W_N^(n2 k1) W_N2^(n2 k2) sum_n1 x[N2 n1 + n2] W_N1^(n1 k1),
// W_L = exp(-2 pi i / L).  Thread (c, t) of a tile holds x[N2 n1 + t], n1 < N1, of column c,
// takes the N1-point DFT in registers and multiplies by W_N^(t k1).  After one exchange
// through shared memory it holds Y[k1][n2] for k1 = t + N2 q (q < N1/N2) and every n2, and
// the N2-point DFTs in registers give X[k1 + N1 k2].  The inverse runs the same steps
// backwards from that register layout (N2-point inverse DFTs, W_N^(-n2 k1), one exchange,
// N1-point inverse DFT), so the periodic z solve (forward transform, division, inverse
// transform) needs two exchanges in all and ends in the layout it was loaded in.
//
// Tiles of B consecutive kx columns by N rows arrive by TMA (tma_pipe.cuh) in one of two
// shared-memory buffers of a persistent CTA while the other tile is transformed; the twiddle
// table W_N^j (and, for the z solve, the eigenvalues along z) is staged in shared memory once.  Once a
// tile sits in registers its buffer is the exchange area: column c at offset c xp, entry
// (k1, n2) at k1 (N2 + 1) + n2, with xp chosen so that neither exchange has bank conflicts.
// Results go from registers straight to HBM, B consecutive complex values per row.
#include "flups_impl.cuh"
#include "regfft.cuh"
#include "tma_pipe.cuh"

namespace {

// ------------------------------------------------ the column kernel
// Threads per CTA: B N2 = 128 (256 for N = 256, where B = 16); the launch bounds hold the
// registers to what three (N >= 512), two (N = 256) or four CTAs per SM allow, the number
// that fits the two tile buffers in shared memory.
// KIND 0: transform along y (INV: inverse).  KIND 1: periodic z solve: forward transform,
// division by lam_x + lam_y + lam_z (the tables hold eigenvalues times the transforms'
// normalisation; the (0, 0, 0) mode, lam = 0, is set to zero), inverse transform.
// tw[j] = W_N^j, j < N.  xp: column pitch of the exchange area (complex values); buf_bytes:
// bytes of each of the two buffers (tile and exchange area, 128-byte multiple).
template <int N1, int N2, int KIND, bool INV>
__global__ void __launch_bounds__(N1 * N2 == 256 ? 256 : 128, N1 * N2 == 256 ? 2 : (N1 * N2 >= 512 ? 3 : 4)) k_cols4(float2* __restrict__ S, const __grid_constant__ CUtensorMap tm, Geo g,
                                               const float2* __restrict__ tw, const float* __restrict__ lamx,
                                               const float* __restrict__ lamy, const float* __restrict__ lamz,
                                               int lgB, int box_rows, int xp, unsigned buf_bytes,
                                               int* __restrict__ err) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    constexpr int N = N1 * N2, Q = N1 / N2;
    constexpr bool FWD_INV = KIND == 0 ? INV : false;   // direction of the first transform
    extern __shared__ __align__(128) unsigned char smc[];
    const int B = 1 << lgB;
    const size_t rs = KIND == 0 ? (size_t)g.ldS : (size_t)g.ny * g.ldS;    // row stride (complex values)
    const int tiles_x = g.M >> lgB;
    const int ntiles = tiles_x * (KIND == 0 ? g.nz : g.ny);
    const unsigned tile_bytes = (unsigned)(N * B * sizeof(float2));
    // after the two buffers: the twiddles W_N^j and (z solve) the eigenvalues lam_z, staged once
    float2* tws = reinterpret_cast<float2*>(smc + 2 * (size_t)buf_bytes);
    float* lzs = reinterpret_cast<float*>(tws + N);
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smc + 2 * (size_t)buf_bytes +
                                                                    (size_t)N * (KIND == 1 ? 12 : 8));
    const int tid = threadIdx.x;
    const int c = tid & (B - 1), t = tid >> lgB;

    auto buffer = [&](int b) { return reinterpret_cast<float2*>(smc + (size_t)b * buf_bytes); };
    auto issue = [&](int tile, int b) {      // one thread: expect the tile's bytes, then TMA its boxes
        if (tid == 0) {
            float2* dst = buffer(b);
            const int tx = tile % tiles_x, ty = tile / tiles_x;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&mbar[b], tile_bytes);
            for (int r0 = 0; r0 < N; r0 += box_rows) {
                if (KIND == 0) tma_load_3d(dst + r0 * B, &tm, tx * B, r0, ty, &mbar[b]);
                else tma_load_3d(dst + r0 * B, &tm, tx * B, ty, r0, &mbar[b]);
            }
        }
    };

    if (smem_u32(smc) & 127u) {   // TMA box destinations must be 128-byte aligned
        if (tid == 0) atomicExch(err, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int j = tid; j < N; j += blockDim.x) {
        tws[j] = __ldg(&tw[j]);
        if (KIND == 1) lzs[j] = __ldg(&lamz[j]);
    }
    __syncthreads();
    unsigned parity[2] = {0u, 0u};
    int tile = blockIdx.x;
    if (tile < ntiles) issue(tile, 0);
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int b = it & 1;
        const int tn = tile + gridDim.x;
        if (tn < ntiles) issue(tn, b ^ 1);
        const bool ok = __syncthreads_and(mbar_wait_bounded(&mbar[b], parity[b]));
        parity[b] ^= 1u;
        if (!ok) {   // leave only after (bounded) waits for both buffers' copies
            if (tid == 0) atomicExch(err, 1);
            mbar_wait_bounded(&mbar[b], parity[b] ^ 1u);
            if (tn < ntiles) mbar_wait_bounded(&mbar[b ^ 1], parity[b ^ 1]);
            return;
        }
        float2* s = buffer(b);
        const int tx = tile % tiles_x, ty = tile / tiles_x;

        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = s[(N2 * n1 + t) * B + c];
        __syncthreads();                       // tile consumed: the buffer becomes the exchange area
        RegDft<N1, FWD_INV>::run(v);
        {
            int idx = 0;                       // W_N^(t k1)
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) {
                idx = (idx + t) & (N - 1);
                v[k1] = tmul<FWD_INV>(v[k1], tws[idx]);
            }
        }
        float2* X = s + c * xp;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) X[k1 * (N2 + 1) + t] = v[k1];
        __syncthreads();
        float2 u[Q][N2];
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) u[q][n2] = X[(t + N2 * q) * (N2 + 1) + n2];
#pragma unroll
        for (int q = 0; q < Q; ++q) RegDft<N2, FWD_INV>::run(u[q]);
        float2* col = (KIND == 0 ? S + (size_t)ty * g.ny * g.ldS : S + (size_t)ty * g.ldS) + (size_t)tx * B + c;
        if (KIND == 0) {
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) col[(size_t)(t + N2 * q + N1 * k2) * rs] = u[q][k2];
        } else {
            const float lxy = __ldg(&lamx[tx * B + c]) + __ldg(&lamy[ty]);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) {
                    const float lam = lxy + lzs[t + N2 * q + N1 * k2];
                    const float inv = lam != 0.f ? rcp_approx(lam) : 0.f;
                    u[q][k2].x *= inv;
                    u[q][k2].y *= inv;
                }
                RegDft<N2, true>::run(u[q]);
                const int k1 = t + N2 * q;      // W_N^(-n2 k1)
                int idx = 0;
#pragma unroll
                for (int n2 = 1; n2 < N2; ++n2) {
                    idx = (idx + k1) & (N - 1);
                    u[q][n2] = tmul<true>(u[q][n2], tws[idx]);
                }
            }
            __syncthreads();                   // every thread has read the first exchange
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int n2 = 0; n2 < N2; ++n2) X[(t + N2 * q) * (N2 + 1) + n2] = u[q][n2];
            __syncthreads();
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) v[k1] = X[k1 * (N2 + 1) + t];
            RegDft<N1, true>::run(v);
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) col[(size_t)(N2 * n1 + t) * rs] = v[n1];
        }
        // this thread's last generic access to the buffer is ordered before the TMA that
        // refills it (issued by thread 0 after the barrier)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
}

// Exchange pitch: at least N1 (N2 + 1), and = 16/B (B <= 16) modulo 16 so that the sixteen
// 8-byte accesses of each half-warp (B columns times 16/B consecutive t) fall in distinct
// bank pairs in both directions of both exchanges.
int cols4_xp(int N1, int N2, int B) {
    const int need = N1 * (N2 + 1);
    const int r = B >= 16 ? 1 : 16 / B;
    int xp = need;
    while (xp % 16 != r % 16) ++xp;
    return xp;
}

template <int N1, int N2, int KIND, bool INV>
cudaError_t launch_k(flups_plan P, float2* S, const Geo& g, int lgB) {
    constexpr int N = N1 * N2;
    const int B = 1 << lgB;
    const int xp = cols4_xp(N1, N2, B);
    size_t bytes = (size_t)N * B * sizeof(float2);
    const size_t xbytes = (size_t)B * xp * sizeof(float2);
    if (xbytes > bytes) bytes = xbytes;
    const unsigned buf_bytes = (unsigned)((bytes + 127) / 128 * 128);
    const size_t sm = 2 * (size_t)buf_bytes + (size_t)N * (KIND == 1 ? 12 : 8) + 2 * sizeof(unsigned long long);
    const int threads = B * N2;
    auto kern = k_cols4<N1, N2, KIND, INV>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int nsm = 0, dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm);
    if (per_sm < 1) per_sm = 1;
    const int ntiles = (g.M / B) * (KIND == 0 ? g.nz : g.ny);
    const int grid = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;
    const float2* tw = (const float2*)(KIND == 0 ? P->twy : P->twz);
    kern<<<grid, threads, sm, P->stream>>>(S, KIND == 0 ? P->tm_y : P->tm_z, g, tw, (const float*)P->lamx,
                                           (const float*)P->lamy, (const float*)P->lamz, lgB, N < 256 ? N : 256, xp,
                                           buf_bytes, &P->sc->err);
    return cudaGetLastError();
}

template <int N1, int N2>
cudaError_t launch_n(flups_plan P, float2* S, const Geo& g, int lgB, int kind, bool inv) {
    if (kind == 1) return launch_k<N1, N2, 1, false>(P, S, g, lgB);
    return inv ? launch_k<N1, N2, 0, true>(P, S, g, lgB) : launch_k<N1, N2, 0, false>(P, S, g, lgB);
}

}  // namespace

// Tile width (log2) of the four-step column kernel for length N and M = nx/2 columns (kind 0:
// y transform, 1: periodic z solve), or -1 when it does not apply: N a power of two in
// [64, 1024]; B the largest of 16, 8, 4, 2 that divides M with a tile of at most 32 KB
// (B N <= 4096; measured at N = 512 along y and z: B = 8 beats 4 and 2).
int cols4_lgB(int N, int M, int kind) {
    if (N < 64 || N > 1024 || (N & (N - 1)) != 0) return -1;
    (void)kind;                                  // the same tile rule along y and z
    for (int B = 16; B >= 2; B >>= 1)
        if (B * N <= 4096 && B <= M && M % B == 0) {
            int l = 0;
            while ((1 << l) < B) ++l;
            return l;
        }
    return -1;
}

bool launch_cols4(flups_plan P, float2* S, const Geo& g, int kind, bool inv) {
    const int N = kind == 0 ? g.ny : g.nz;
    const int lgB = cols4_lgB(N, g.M, kind);
    if (lgB < 0) return false;
    switch (N) {
        case 64: launch_n<8, 8>(P, S, g, lgB, kind, inv); break;
        case 128: launch_n<16, 8>(P, S, g, lgB, kind, inv); break;
        case 256: launch_n<16, 16>(P, S, g, lgB, kind, inv); break;
        case 512: launch_n<32, 16>(P, S, g, lgB, kind, inv); break;
        default: launch_n<32, 32>(P, S, g, lgB, kind, inv); break;
    }
    return true;
}

namespace {

// ------------------------------------------------ z walls: partitioned Gauss elimination
// The tridiagonal system of column (kx, ky) (Sec. 3.3.1, step 5),
//     a_k P_{k-1} + (b_k + lam) P_k + c_k P_{k+1} = F_k,   lam = lam_x(kx) + lam_y(ky),
// solved without any HBM scratch: a tile of B consecutive kx columns by nz rows arrives by
// TMA in shared memory, and thread (c, q) of the CTA takes rows [q MC, q MC + MC) of column c
// (at most 32 chunks).  The last row of every chunk but the last is a separator; the other
// rows of chunk q (its interior) depend only on the separators E_{q-1} below and E_q above,
// and a Thomas sweep in registers gives them as P_k = y_k + al_k E_{q-1} + be_k E_q.
// Substituting the interior rows next to each separator into the separator's own row gives a
// tridiagonal system of at most 31 unknowns, A_j E_{j-1} + D_j E_j + C_j E_{j+1} = G_j, which
// one warp per column solves by parallel cyclic reduction on warp shuffles (lane j holds
// equation j; five halving steps eliminate the neighbours at distance 1, 2, 4, 8, 16).  Then
// every thread forms its rows and stores them.  The matrix is weakly diagonally dominant
// (b_k = -(a_k + c_k), lam <= 0), so neither step pivots.  The singular column
// (kx, ky) = (0, 0) of a plan without Dirichlet ends is left to k_ztri_sing.
constexpr int ZNBUF = 3;

template <int MC>
__global__ void __launch_bounds__(256, MC <= 8 ? 3 : 2) k_ztri_tile(float2* __restrict__ S,
                                                                    const __grid_constant__ CUtensorMap tm, Geo g,
                                                                    const float* __restrict__ lamx,
                                                                    const float* __restrict__ lamy,
                                                                    const float* __restrict__ tri, int lgB, int nchunk,
                                                                    int box_rows, int nbox, unsigned buf_bytes,
                                                                    int* __restrict__ err) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    extern __shared__ __align__(128) unsigned char smc[];
    const int B = 1 << lgB, nz = g.nz;
    const int tiles_x = (g.nxh + B - 1) >> lgB;     // the last tile holds the Nyquist column
    const int ntiles = tiles_x * g.ny;
    const unsigned tile_bytes = (unsigned)nbox * box_rows * B * sizeof(float2);
    // shared memory: [ZNBUF tiles][per column c, 33 slots per chunk: yF yL E (complex),
    // aF bF aL bL (real)][mbarriers]: a ring of ZNBUF tile buffers, ZNBUF - 1 tiles in flight
    // while one is solved (enough bytes in flight per SM for HBM latency with 16 KB tiles)
    constexpr int RP = 33;
    float2* rc = reinterpret_cast<float2*>(smc + ZNBUF * (size_t)buf_bytes);
    const int NQ = B * RP;
    float2* yF = rc;             // y of the first and last interior row of each chunk
    float2* yL = rc + NQ;
    float2* Es = rc + 2 * NQ;    // the separators
    float* rr = reinterpret_cast<float*>(rc + 3 * NQ);
    float* aF = rr;              // al, be of the first and last interior rows
    float* bF = rr + NQ;
    float* aL = rr + 2 * NQ;
    float* bL = rr + 3 * NQ;
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smc + ZNBUF * (size_t)buf_bytes +
                                                                    (size_t)NQ * (3 * sizeof(float2) + 4 * sizeof(float)));
    const int tid = threadIdx.x;
    const int c = tid & (B - 1), q = tid >> lgB;
    const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const float* ta = tri;
    const float* tb = tri + nz;
    const float* tc = tri + 2 * nz;
    const int r0 = q * MC;
    const int mi = q < nchunk - 1 ? MC - 1 : nz - r0;   // interior rows of this chunk (>= 1)
    const int nsep = nchunk - 1;

    auto buffer = [&](int b) { return reinterpret_cast<float2*>(smc + (size_t)b * buf_bytes); };
    auto issue = [&](int tile, int b) {
        if (tid == 0) {
            float2* dst = buffer(b);
            const int tx = tile % tiles_x, ty = tile / tiles_x;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&mbar[b], tile_bytes);
            for (int k = 0; k < nbox; ++k) tma_load_3d(dst + k * box_rows * B, &tm, tx * B, ty, k * box_rows, &mbar[b]);
        }
    };

    if (smem_u32(smc) & 127u) {
        if (tid == 0) atomicExch(err, 2);
        return;
    }
    if (tid == 0) {
        for (int k = 0; k < ZNBUF; ++k) mbar_init(&mbar[k], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0u;                  // bit k: phase of buffer k's next completion
    for (int k = 0; k < ZNBUF - 1; ++k)
        if (blockIdx.x + k * (int)gridDim.x < ntiles) issue(blockIdx.x + k * gridDim.x, k);
    int tile = blockIdx.x;
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int b = it % ZNBUF;
        const int tn = tile + (ZNBUF - 1) * gridDim.x;
        if (tn < ntiles) issue(tn, (it + ZNBUF - 1) % ZNBUF);
        const bool ok = __syncthreads_and(mbar_wait_bounded(&mbar[b], (parity >> b) & 1u));
        parity ^= 1u << b;
        if (!ok) {   // leave only after (bounded) waits for every copy this CTA has in flight
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(&mbar[b], ((parity >> b) & 1u) ^ 1u);
                for (int k = 1; k < ZNBUF; ++k) {
                    const int bk = (it + k) % ZNBUF;
                    if (tile + k * (int)gridDim.x < ntiles) mbar_wait_bounded(&mbar[bk], (parity >> bk) & 1u);
                }
            }
            return;
        }
        const float2* s = buffer(b);
        const int tx = tile % tiles_x, ky = tile / tiles_x;
        const float lyk = __ldg(&lamy[ky]);
        const int kx = tx * B + c;
        const bool live = kx < g.nxh && !(g.sing00 && kx == 0 && ky == 0);
        const float lam = __ldg(&lamx[kx < g.nxh ? kx : 0]) + lyk;

        // interior rows: Thomas sweep with the right-hand sides F, -a e_first (left separator)
        // and -c e_last (right separator); the previous row's values ride in scalars
        float cp[MC], al[MC], be[MC];
        float2 y[MC];
        {
            float cprev = 0.f, aprev = 0.f;
            float2 yprev = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < MC; ++i) {
                if (i < mi) {
                    const int r = r0 + i;
                    const float a = __ldg(&ta[r]);
                    const float inv = rcp_approx((__ldg(&tb[r]) + lam) - a * cprev);
                    const float cr = __ldg(&tc[r]) * inv;
                    const float2 F = s[r * B + c];
                    yprev = make_float2((F.x - a * yprev.x) * inv, (F.y - a * yprev.y) * inv);
                    aprev = (i == 0 ? -a : -a * aprev) * inv;
                    cprev = cr;
                    y[i] = yprev;
                    al[i] = aprev;
                    cp[i] = cr;                       // unused at the last interior row
                    be[i] = -cr;                      // the right separator's column (last row only)
                }
            }
        }
        float2 ylast = make_float2(0.f, 0.f), ynext = make_float2(0.f, 0.f);
        float alast = 0.f, blast = 0.f, anext = 0.f, bnext = 0.f;
#pragma unroll
        for (int i = MC - 1; i >= 0; --i) {
            if (i < mi) {
                if (i < mi - 1) {                     // back substitution
                    y[i].x -= cp[i] * ynext.x;
                    y[i].y -= cp[i] * ynext.y;
                    al[i] -= cp[i] * anext;
                    be[i] = -cp[i] * bnext;
                } else {
                    ylast = y[i];
                    alast = al[i];
                    blast = be[i];
                }
                ynext = y[i];
                anext = al[i];
                bnext = be[i];
            }
        }
        {
            const int o = c * RP + q;
            yF[o] = y[0];
            aF[o] = al[0];
            bF[o] = be[0];
            yL[o] = ylast;
            aL[o] = alast;
            bL[o] = blast;
        }
        __syncthreads();
        // separators: one warp per column, parallel cyclic reduction on shuffles
        if (nsep > 0) {
            for (int cc = warp; cc < B; cc += nwarp) {
                const int kxc = tx * B + cc;
                const float lamc = __ldg(&lamx[kxc < g.nxh ? kxc : 0]) + lyk;
                float A = 0.f, D = 1.f, C = 0.f;
                float2 G = make_float2(0.f, 0.f);
                if (lane < nsep) {
                    const int r = lane * MC + MC - 1, o = cc * RP + lane;
                    const float a = __ldg(&ta[r]), cz = __ldg(&tc[r]);
                    A = a * aL[o];
                    D = a * bL[o] + (__ldg(&tb[r]) + lamc) + cz * aF[o + 1];
                    C = cz * bF[o + 1];
                    const float2 F = s[r * B + cc];
                    G = make_float2(F.x - a * yL[o].x - cz * yF[o + 1].x, F.y - a * yL[o].y - cz * yF[o + 1].y);
                }
#pragma unroll
                for (int st = 1; st < 32; st <<= 1) {
                    float Am = __shfl_up_sync(0xffffffffu, A, st), Dm = __shfl_up_sync(0xffffffffu, D, st);
                    float Cm = __shfl_up_sync(0xffffffffu, C, st);
                    float Gmx = __shfl_up_sync(0xffffffffu, G.x, st), Gmy = __shfl_up_sync(0xffffffffu, G.y, st);
                    float Ap = __shfl_down_sync(0xffffffffu, A, st), Dp = __shfl_down_sync(0xffffffffu, D, st);
                    float Cq = __shfl_down_sync(0xffffffffu, C, st);
                    float Gpx = __shfl_down_sync(0xffffffffu, G.x, st), Gpy = __shfl_down_sync(0xffffffffu, G.y, st);
                    if (lane < st) { Am = 0.f; Dm = 1.f; Cm = 0.f; Gmx = 0.f; Gmy = 0.f; }        // identity rows
                    if (lane + st >= 32) { Ap = 0.f; Dp = 1.f; Cq = 0.f; Gpx = 0.f; Gpy = 0.f; }
                    const float alpha = -A * rcp_approx(Dm), gamma = -C * rcp_approx(Dp);
                    D = D + alpha * Cm + gamma * Ap;
                    G = make_float2(G.x + alpha * Gmx + gamma * Gpx, G.y + alpha * Gmy + gamma * Gpy);
                    A = alpha * Am;
                    C = gamma * Cq;
                }
                if (lane < nsep) {
                    const float inv = rcp_approx(D);
                    Es[cc * RP + lane] = make_float2(G.x * inv, G.y * inv);
                }
            }
        }
        __syncthreads();
        if (live) {
            const float2 EL = q > 0 ? Es[c * RP + q - 1] : make_float2(0.f, 0.f);
            const float2 ER = q < nchunk - 1 ? Es[c * RP + q] : make_float2(0.f, 0.f);
            float2* col = S + (size_t)ky * g.ldS + kx;
            const size_t zs = (size_t)g.ny * g.ldS;
#pragma unroll
            for (int i = 0; i < MC; ++i) {
                if (i < mi)
                    col[(size_t)(r0 + i) * zs] = make_float2(y[i].x + al[i] * EL.x + be[i] * ER.x,
                                                             y[i].y + al[i] * EL.y + be[i] * ER.y);
            }
            if (q < nchunk - 1) col[(size_t)(r0 + MC - 1) * zs] = ER;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
}

// The singular column (kx, ky) = (0, 0) of a walls plan without Dirichlet ends (one CTA):
// the dzf-weighted mean of F is removed (so that dropping row 0 solves L p = f - <f>_V for any
// f), row 0 is dropped with P_0 = 0, rows 1..nz-1 are solved by Thomas, and the column is
// shifted to zero dzf-weighted mean.  The column is staged in shared memory (F, then the
// multipliers), the sweeps run on one thread.
__global__ void __launch_bounds__(256) k_ztri_sing(float2* __restrict__ S, Geo g, const float* __restrict__ tri) {
    if (g.skip && *g.skip) return;
    extern __shared__ __align__(16) unsigned char sms[];
    const int nz = g.nz;
    float2* x = reinterpret_cast<float2*>(sms);
    float* cps = reinterpret_cast<float*>(x + nz);
    __shared__ double red[3][8];
    const size_t zs = (size_t)g.ny * g.ldS;
    double sw = 0.0, sx = 0.0, sy = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const float2 F = S[(size_t)k * zs];
        x[k] = F;
        const double w = g.dzf[k];
        sw += w;
        sx += w * (double)F.x;
        sy += w * (double)F.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_down_sync(0xffffffffu, sw, o);
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sw;
        red[1][threadIdx.x >> 5] = sx;
        red[2][threadIdx.x >> 5] = sy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tw = 0.0, tx = 0.0, ty = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tw += red[0][w]; tx += red[1][w]; ty += red[2][w]; }
        const float mx = (float)(tx / tw), my = (float)(ty / tw);
        const float* ta = tri;
        const float* tb = tri + nz;
        const float* tc = tri + 2 * nz;
        float cprev = 0.f;
        float2 dprev = make_float2(0.f, 0.f);
        for (int k = 1; k < nz; ++k) {
            const float a = k > 1 ? ta[k] : 0.f;
            const float inv = 1.f / (tb[k] - a * cprev);
            cprev = tc[k] * inv;
            cps[k] = cprev;
            const float2 F = x[k];
            dprev = make_float2(((F.x - mx) - a * dprev.x) * inv, ((F.y - my) - a * dprev.y) * inv);
            x[k] = dprev;
        }
        float2 xv = x[nz - 1];
        double px = (double)g.dzf[nz - 1] * xv.x, py = (double)g.dzf[nz - 1] * xv.y;
        for (int k = nz - 2; k >= 1; --k) {
            const float2 d = x[k];
            xv = make_float2(d.x - cps[k] * xv.x, d.y - cps[k] * xv.y);
            x[k] = xv;
            px += (double)g.dzf[k] * xv.x;
            py += (double)g.dzf[k] * xv.y;
        }
        x[0] = make_float2(0.f, 0.f);
        red[0][0] = px / tw;
        red[1][0] = py / tw;
    }
    __syncthreads();
    const float mx = (float)red[0][0], my = (float)red[1][0];
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const float2 v = x[k];
        S[(size_t)k * zs] = make_float2(v.x - mx, v.y - my);
    }
}

// Layout of the walls tile kernel for nz rows: rows per chunk MC (the power of two >= nz/32,
// at least 2, at most 16: at most 32 chunks, so the separators fit one warp), chunks per
// column, tile width B (the largest power of two <= 16 with at most 256 threads), box rows and
// boxes per tile.  False where it does not apply (nz > 512).
bool ztri_layout(int nz, int* mc, int* nchunk, int* lgB, int* box_rows, int* nbox) {
    if (nz < 2 || nz > 512) return false;
    int m = 2;
    while (m * 32 < nz) m <<= 1;
    if (m > 16) return false;                   // instantiated for 2, 4, 8, 16 rows per chunk
    *mc = m;
    *nchunk = (nz + m - 1) / m;
    int B = 16;
    while (B > 2 && B * *nchunk > 256) B >>= 1;
    if (B * *nchunk > 256) return false;
    int l = 0;
    while ((1 << l) < B) ++l;
    *lgB = l;
    *box_rows = nz < 256 ? nz : 256;
    *nbox = (nz + *box_rows - 1) / *box_rows;
    return true;
}

template <int MC>
void launch_ztri_mc(flups_plan P, float2* S, const Geo& g, int nchunk, int lgB, int box_rows, int nbox) {
    const int B = 1 << lgB;
    const unsigned buf_bytes = (unsigned)(((size_t)nbox * box_rows * B * sizeof(float2) + 127) / 128 * 128);
    const size_t red = (size_t)33 * B * (3 * sizeof(float2) + 4 * sizeof(float));
    const size_t sm = ZNBUF * (size_t)buf_bytes + (red + 15) / 16 * 16 + ZNBUF * sizeof(unsigned long long);
    auto kern = k_ztri_tile<MC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int nsm = 0, dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = B * nchunk;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm);
    if (per_sm < 1) per_sm = 1;
    const int ntiles = ((g.nxh + B - 1) / B) * g.ny;
    const int grid = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;
    kern<<<grid, threads, sm, P->stream>>>(S, P->tm_z, g, (const float*)P->lamx, (const float*)P->lamy,
                                           (const float*)P->tri, lgB, nchunk, box_rows, nbox, buf_bytes, &P->sc->err);
}

}  // namespace

int ztri_tile_lgB(int nz) {
    int mc, nchunk, lgB, box_rows, nbox;
    return ztri_layout(nz, &mc, &nchunk, &lgB, &box_rows, &nbox) ? lgB : -1;
}

int launch_ztri_tile(flups_plan P, float2* S, const Geo& g) {
    int mc, nchunk, lgB, box_rows, nbox;
    if (!P->tma_ok || !ztri_layout(g.nz, &mc, &nchunk, &lgB, &box_rows, &nbox)) return 0;
    switch (mc) {
        case 2: launch_ztri_mc<2>(P, S, g, nchunk, lgB, box_rows, nbox); break;
        case 4: launch_ztri_mc<4>(P, S, g, nchunk, lgB, box_rows, nbox); break;
        case 8: launch_ztri_mc<8>(P, S, g, nchunk, lgB, box_rows, nbox); break;
        default: launch_ztri_mc<16>(P, S, g, nchunk, lgB, box_rows, nbox); break;
    }
    int n = 1;
    if (g.sing00) {
        const size_t sm = (size_t)g.nz * (sizeof(float2) + sizeof(float));
        cudaFuncSetAttribute(k_ztri_sing, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_ztri_sing<<<1, 256, sm, P->stream>>>(S, g, (const float*)P->tri);
        n = 2;
    }
    return n;
}
