// pnet.cu - learned splitting pressure: a periodic 3-D convolutional net that predicts the
// correction to the linear extrapolation p_hat = 2 p^n - p^{n-1} of Sec. 3.3, trained on the
// exact variable-coefficient pressures of flups_varcoef_solve.
//
//   features  x = (1 - rho0/rho, p^n/s, p^{n-1}/s), s = rms(p^n)
//   net       four 3x3x3 convolutions 3 -> 16 -> 16 -> 16 -> 1, ReLU between layers
//   output    p_hat = 2 p^n - p^{n-1} + s y
//   training  loss = mean (y - (p^{n+1} - 2 p^n + p^{n-1})/s)^2, Adam (beta 0.9/0.999, eps 1e-8)
//
// Arithmetic: every convolution is an implicit GEMM on the tensor cores (mma.sync m16n8k16,
// bfloat16 operands, FP32 accumulation).  Activations and gradients are stored as bfloat16
// [point][16 channels] (32 bytes a point, channels fastest); master weights, Adam moments and
// gradients are FP32; biases are added in FP32.
//
// A CTA computes a tile of 4 (z) x 8 (y) x 32 (x) output points from a shared-memory halo tile
// of 6 x 10 x 34 input points.  The 16-byte halves of a point are stored swapped when bit 2 of
// the point's tile index is set, so the eight 16-byte rows an ldmatrix reads for eight
// consecutive points fall in eight different bank groups.
//
// Packed weights (per layer, bfloat16 [27 taps][16 rows][24]): the forward form has rows = output
// channel and columns = input channel; the backward-data form of layer l has rows = input
// channel, columns = output channel and the taps reversed (tap t -> 26 - t), so the gradient
// with respect to a layer's input is the same convolution kernel run on the output gradient.
// Padding columns/rows are zero.
//
// On grids with nx a multiple of 128 the convolutions run on the 5th-generation tensor cores
// instead (k_pnet_conv_tcz), and on grids of nx = 64 the output layer does (k_pnet_conv_tcz64:
// two y rows of 64 points per MMA, from dx-rotated copies of each input row; the 16-channel
// layers measured faster on mma.sync there).  In k_pnet_conv_tcz each MMA computes 128
// consecutive x-points of one input row against the 16 output channels of up to three output
// rows (N = 16, 32 or 48: the row's dy taps) with K = 16 input channels (tcgen05.mma kind::f16,
// bf16 operands from shared memory, FP32 accumulators in tensor memory); the taps accumulate
// into the same tensor-memory columns.  The A operand is read straight out of the halo tile with
// one descriptor per input row and x shift: the tile stores each point's two 8-channel halves in
// two planes (point stride 16 bytes), so an x-shifted window of 128 points is again a K-major
// operand (core matrices of 8 points x 16 bytes 128 bytes apart, the two K halves one plane
// apart).  Loads, MMAs and the epilogue run in separate warps, linked by mbarriers.

#include "flups_impl.cuh"

#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#define PN_NP 15601
#define PN_WPK (27 * 16 * 24)          // packed weights of one layer (bf16 elements)
#define PN_PART 6928                   // one CTA's weight-gradient partial: 27*16*16 + 16 biases
#define PN_TCW (27 * 256)              // tcgen05-layout weights of one layer (bf16 elements)

namespace {

constexpr int TZ = 4, TY = 8, TX = 32;
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2;
constexpr int NHALO = HZ * HY * HX;                       // 2040 points
constexpr int TILE_PTS = TZ * TY * TX;                    // 1024 points
constexpr int SMEM_IN = NHALO * 32;                       // 65280 bytes
constexpr int SMEM_W = PN_WPK * 2;                        // 20736 bytes
constexpr int SMEM_DZ = TILE_PTS * 32;                    // 32768 bytes
constexpr int CONV_SMEM = SMEM_IN + SMEM_W;
constexpr int WGRAD_SMEM = SMEM_IN + SMEM_DZ;
constexpr int THREADS = 256;

// layer geometry: inputs, outputs, offsets of W and b in the parameter vector
__host__ __device__ constexpr int lay_in(int l) { return l == 0 ? 3 : 16; }
__host__ __device__ constexpr int lay_out(int l) { return l == 3 ? 1 : 16; }
__host__ __device__ constexpr int lay_w(int l) { return l == 0 ? 0 : (l == 1 ? 1312 : (l == 2 ? 8240 : 15168)); }
__host__ __device__ constexpr int lay_b(int l) { return lay_w(l) + lay_out(l) * lay_in(l) * 27; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// byte offset of 16-byte half h of tile point sp (swizzled)
__device__ __forceinline__ uint32_t swz(int sp, int h) { return (uint32_t)((sp * 2 + (h ^ ((sp >> 2) & 1))) * 16); }

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

struct TileOrigin { int x0, y0, z0; };

__device__ __forceinline__ TileOrigin tile_origin(int nx, int ny) {
    const int tnx = nx / TX, tny = ny / TY;
    const int b = blockIdx.x;
    TileOrigin o;
    o.x0 = (b % tnx) * TX;
    o.y0 = ((b / tnx) % tny) * TY;
    o.z0 = (b / (tnx * tny)) * TZ;
    return o;
}

// Loads the periodic halo tile of a [n][16] bfloat16 field into shared memory (swizzled).
// Loads are issued in batches of 8 per thread before the shared-memory stores.
__device__ __forceinline__ void load_halo(const __nv_bfloat16* __restrict__ in, unsigned char* sm, TileOrigin o,
                                          int nx, int ny, int nz) {
    const uint4* src = reinterpret_cast<const uint4*>(in);
    constexpr int NC = NHALO * 2, BT = 8;
    for (int c0 = threadIdx.x; c0 < NC; c0 += THREADS * BT) {
        uint4 v[BT];
        uint32_t dst[BT];
#pragma unroll
        for (int q = 0; q < BT; ++q) {
            const int c = c0 + q * THREADS;
            if (c < NC) {
                const int sp = c >> 1, h = c & 1;
                const int xx = sp % HX, t = sp / HX;
                const int yy = t % HY, zz = t / HY;
                const int gx = wrapc(o.x0 + xx - 1, nx), gy = wrapc(o.y0 + yy - 1, ny), gz = wrapc(o.z0 + zz - 1, nz);
                const long long pt = ((long long)gz * ny + gy) * nx + gx;
                v[q] = __ldg(src + pt * 2 + h);
                dst[q] = swz(sp, h);
            }
        }
#pragma unroll
        for (int q = 0; q < BT; ++q)
            if (c0 + q * THREADS < NC) *reinterpret_cast<uint4*>(sm + dst[q]) = v[q];
    }
}

struct ConvArgs {
    const __nv_bfloat16* in;     // [n][16]
    const __nv_bfloat16* w;      // packed weights [27][16][24] (mma.sync kernel)
    const __nv_bfloat16* wtc;    // packed weights [27][2 halves][16][8] (tcgen05 kernel)
    int* err;                    // nonzero: a bounded wait of the tcgen05 kernel timed out
    const float* bias;           // FP32 biases (EPI 0, 1, 2)
    __nv_bfloat16* out;          // EPI 0: activation; EPI 2: output gradient (channel 0); EPI 3: masked gradient
    const __nv_bfloat16* mask;   // EPI 3: activation whose positive entries pass the gradient
    const double* pn;            // EPI 1, 2
    const double* pnm1;
    const double* pnext;         // EPI 2
    double* phat;                // EPI 1
    const double* sc;            // [0] s, [1] 1/s
    double* red;                 // EPI 2: per-CTA sum of squared errors
    double gscale;               // EPI 2: d loss / d y = gscale * error
    int nx, ny, nz;
};

// EPI 0: out = bf16(relu(acc + b))           (hidden layer, NT = 2)
// EPI 1: p_hat = 2 p^n - p^{n-1} + s (acc + b) (last layer inference, NT = 1)
// EPI 2: e = acc + b - t, out[.][0] = bf16(gscale e), red += e^2 (last layer training, NT = 1)
// EPI 3: out = bf16(acc * (mask > 0))          (gradient w.r.t. a hidden layer's output, NT = 2)
template <int NT, int EPI>
__global__ void __launch_bounds__(THREADS, 2) k_pnet_conv(ConvArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* sin = sm;
    unsigned char* sw = sm + SMEM_IN;
    const TileOrigin o = tile_origin(a.nx, a.ny);
    load_halo(a.in, sin, o, a.nx, a.ny, a.nz);
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.w);
        const int nchunk = (NT == 2 ? 16 : 8) * 24 * 2 / 16;     // 16-byte chunks per tap (rows used)
        for (int c = threadIdx.x; c < 27 * nchunk; c += THREADS) {
            const int tap = c / nchunk, r = c % nchunk;
            reinterpret_cast<uint4*>(sw)[tap * 48 + r] = __ldg(src + tap * 48 + r);
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int zl = warp >> 1, ybase = (warp & 1) * 4;
    const uint32_t sin_u = smem_u32(sin), sw_u = smem_u32(sw);
    // ldmatrix row of this lane: A operand (points x channels), B operand (weights)
    const int a_row = (lane & 7) + ((lane >> 3) & 1) * 8, a_half = lane >> 4;
    const uint32_t b_off = (uint32_t)((((lane >> 4) * 8 + (lane & 7)) * 24 + ((lane >> 3) & 1) * 8) * 2);
    const int g = lane >> 2, t4 = lane & 3;

    double sq = 0.0;
    for (int grp = 0; grp < 2; ++grp) {
        float acc[4][NT][4];
#pragma unroll
        for (int mi = 0; mi < 4; ++mi)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[mi][nt][q] = 0.0f;
        const int y0l = ybase + 2 * grp;
#pragma unroll 1
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            uint32_t b[4];
            if (NT == 2) {
                ldsm_x4(sw_u + tap * (16 * 24 * 2) + b_off, b);
            } else {
                ldsm_x2(sw_u + tap * (16 * 24 * 2) + b_off, b[0], b[1]);
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int yl = y0l + (mi >> 1), xh = mi & 1;
                const int sp = ((zl + dz + 1) * HY + (yl + dy + 1)) * HX + xh * 16 + dx + 1 + a_row;
                uint32_t av[4];
                ldsm_x4(sin_u + swz(sp, a_half), av);
                mma_bf16(acc[mi][0], av, b[0], b[1]);
                if (NT == 2) mma_bf16(acc[mi][NT - 1], av, b[2], b[3]);
            }
        }
        // epilogue
#pragma unroll
        for (int mi = 0; mi < 4; ++mi) {
            const int yl = y0l + (mi >> 1), xh = mi & 1;
            const long long rowbase = ((long long)(o.z0 + zl) * a.ny + (o.y0 + yl)) * a.nx + o.x0 + xh * 16;
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                const long long pt = rowbase + g + 8 * hr;
                if (EPI == 0 || EPI == 3) {
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) {
                        const int n = nt * 8 + 2 * t4;
                        float v0 = acc[mi][nt][2 * hr], v1 = acc[mi][nt][2 * hr + 1];
                        if (EPI == 0) {
                            v0 = fmaxf(v0 + __ldg(a.bias + n), 0.0f);
                            v1 = fmaxf(v1 + __ldg(a.bias + n + 1), 0.0f);
                        } else {
                            const uint32_t mk = __ldg(reinterpret_cast<const unsigned int*>(a.mask + pt * 16 + n));
                            if (!(mk & 0x7fffu)) v0 = 0.0f;
                            if (!(mk & 0x7fff0000u)) v1 = 0.0f;
                        }
                        *reinterpret_cast<__nv_bfloat162*>(a.out + pt * 16 + n) = __floats2bfloat162_rn(v0, v1);
                    }
                } else if (t4 == 0) {
                    const double y = (double)(acc[mi][0][2 * hr] + __ldg(a.bias));
                    const double pn = a.pn[pt], pm = a.pnm1[pt];
                    if (EPI == 1) {
                        a.phat[pt] = 2.0 * pn - pm + a.sc[0] * y;
                    } else {
                        const double e = y - (a.pnext[pt] - (2.0 * pn - pm)) * a.sc[1];
                        sq += e * e;
                        a.out[pt * 16] = __double2bfloat16(a.gscale * e);
                    }
                }
            }
        }
    }
    if (EPI == 2) {
        __shared__ double ws[THREADS / 32];
        for (int s = 16; s > 0; s >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s);
        if (lane == 0) ws[warp] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < THREADS / 32; ++w) t += ws[w];
            a.red[blockIdx.x] = t;
        }
    }
}

// ------------------------------------------------------------ tcgen05 convolution
// Shared-memory matrix descriptor (no swizzle, K-major): start address, leading byte offset
// (step between the two K halves), stride byte offset (step between 8-row core matrices).
__device__ __forceinline__ unsigned long long tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
constexpr uint32_t TC_IDESC = tc_idesc(16);

__device__ __forceinline__ bool tc_mbar_try(uint32_t m, uint32_t par) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(m), "r"(par) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// tcgen05.ld of 16 columns without the wait; tc_wait16 completes it (the registers pass through
// the wait, so that no use of them is scheduled before it)
__device__ __forceinline__ void tc_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tc_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :: "memory");
}
__device__ __forceinline__ uint32_t tc_ld1_async(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return r;
}
__device__ __forceinline__ void tc_wait4(uint32_t (&r)[4]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) :: "memory");
}

__device__ __forceinline__ float tc_ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}

// tcgen05 convolution marching in z, warp-specialized.  A CTA owns a column of 4 (y) x 128 (x)
// points through zc planes.  Input planes (rows y0-1 .. y0+4, x0-1 .. x0+128, both 8-channel
// halves as planes of 16-byte points) pass through a ring of TW_R shared-memory slots: local input
// i (global plane z0 - 1 + i) sits in slot i mod TW_R, and output plane o reads inputs o, o+1, o+2.
//   warps 1-3 (producers): 16-byte asynchronous copies of input i once slot i mod TW_R is free
//     (mbarrier empty, arrived by the MMAs of plane i - TW_R), then full[slot] when they landed
//     (TW_LAG planes behind their issue: input i - TW_LAG is published after input i is issued,
//     which needs the MMAs of plane i - TW_R, which need input i - TW_R + 2 <= i - TW_LAG - 1;
//     the issuer can then run TW_R - 2 - TW_LAG planes ahead of the MMAs' completion);
//   warp 0 lane 0 (MMA issuer): for plane o, waits for input o + 2 and for accumulator set o mod
//     TW_S to be drained, issues the plane's 54 MMAs, commits to the set's full barrier and to
//     the empty barrier of input o's slot;
//   warps 4-7 (epilogue, one tensor-memory lane quadrant each, one x point per thread): read the
//     set's 4 rows x 16 columns, store the layer output, clear the set, arrive on its empty barrier.
// Each MMA takes one x-shifted input row (A, 128 points x 16 channels) against the weights of
// every output row it feeds: input row ri (y0 - 1 + ri) enters output rows ri - 2 .. ri (those
// inside the tile) through the taps dy = +1, 0, -1, whose accumulators are adjacent 16-column
// blocks, so one MMA of N = 16, 32 or 48 covers them (B: the three dy blocks of one (dz, dx)
// stacked as 48 rows): 54 MMAs per plane (6 rows x 3 dx x 3 dz) instead of 108 of N = 16, and
// half the A-operand reads.  A plane's first MMA clears its accumulator set (a zero A tile, not
// accumulated); every other MMA accumulates.
// Every wait is bounded: on a timeout the CTA stops its roles, lets its copies and MMAs finish,
// and sets a.err.
// PACKX (the first layer, 3 input channels): the input holds at channel 3 (dx + 1) + c the
// feature c of the point x + dx (k_pnet_features_x), so the three x taps are one K = 16 operand (9
// channels used) and a plane takes 18 MMAs (6 rows x 3 dz), against the x-halo-free window.
constexpr int TZ_TY = 4, TZ_HX = 130, TZ_HY = TZ_TY + 2;
constexpr int TZ_PHALF = TZ_HY * TZ_HX * 16;          // one 8-channel half of an input plane (12480 B)
constexpr int TZ_PLANE = 2 * TZ_PHALF;                // 24960 B
constexpr int TZ_WQ = 1536;                           // weights of one (dz, dx): 2 K halves x 48 rows
constexpr int TZ_THREADS = 256;
constexpr int TW_R = 8;                               // input ring slots
constexpr int TW_S = 4;                               // accumulator sets (4 rows x 16 columns)
constexpr int TW_PROD = 96;                           // producer threads (warps 1-3)
constexpr int TW_LAG = 3;                             // planes between a copy's issue and its publication
static_assert(TW_LAG >= 1 && TW_R - 2 - TW_LAG >= 1, "the producer must publish an input before it waits on "
                                                     "the MMAs that read it");
constexpr int TW_NBAR = 2 * TW_R + 2 * TW_S;          // full, empty, set full, set empty
constexpr int TW_ZERO = 4096;                         // a zero A operand (128 points x 16 channels)
constexpr int TZ_SMEM = TW_R * TZ_PLANE + 27 * 512 + TW_ZERO + TW_NBAR * 8 + 16;
constexpr int TZ_TMEM_COLS = TW_S * 64;
constexpr int TW_CPT = (TZ_HY * TZ_HX * 2 + TW_PROD - 1) / TW_PROD;   // copies per producer thread

template <int EPI, bool PACKX>
__global__ void __launch_bounds__(TZ_THREADS, 1) k_pnet_conv_tcz(ConvArgs a, int zc) {
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* sw = sm + TW_R * TZ_PLANE;
    unsigned char* zt = sw + 27 * 512;                         // zero tile
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(zt + TW_ZERO);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + TW_NBAR);
    __shared__ int abort_;
    __shared__ double ws[4];
    constexpr int FULL = 0, EMPTY = TW_R, SETF = 2 * TW_R, SETE = 2 * TW_R + TW_S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tnx = a.nx / 128, tny = a.ny / TZ_TY;
    const int b = blockIdx.x;
    const int x0 = (b % tnx) * 128, y0 = ((b / tnx) % tny) * TZ_TY, z0 = (b / (tnx * tny)) * zc;
    const uint4* src = reinterpret_cast<const uint4*>(a.in);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TZ_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_ = 0;
        for (int i = 0; i < TW_NBAR; ++i) {
            const int cnt = i < TW_R ? TW_PROD : (i < SETE ? 1 : 4);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar + i)), "r"(cnt) : "memory");
        }
    }
    if (!PACKX) {
        // 16-byte chunk (tap, K half kh, output channel oc) of [27][2][16][8] goes to block
        // i = 1 - dy of the 48-row operand of (dz, dx): [9 (dz, dx)][2 kh][3 i][16 oc] chunks
        const uint4* wsrc = reinterpret_cast<const uint4*>(a.wtc);
        for (int c = tid; c < 27 * 32; c += TZ_THREADS) {
            const int tap = c >> 5, kh = (c >> 4) & 1, oc = c & 15;
            const int q = (tap / 9) * 3 + tap % 3, i = 2 - (tap / 3) % 3;
            reinterpret_cast<uint4*>(sw)[q * (TZ_WQ / 16) + kh * 48 + i * 16 + oc] = __ldg(wsrc + c);
        }
    } else {
        // operand of dz (block i = 1 - dy, K half kh, output channel oc): element k = 8 kh + j is
        // W(dz, dy, dx = k / 3 - 1; oc, c = k % 3) for k < 9, else 0; [3 dz][2 kh][3 i][16 oc] chunks
        const unsigned short* wsrc = reinterpret_cast<const unsigned short*>(a.wtc);
        for (int c = tid; c < 3 * 96; c += TZ_THREADS) {
            const int q = c / 96, kh = (c / 48) & 1, i = (c / 16) % 3, oc = c & 15;
            const int dy = 1 - i;
            uint32_t h[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                uint32_t v2 = 0;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int k = 8 * kh + 2 * jj + hh;
                    if (k < 9) {
                        const int tap = q * 9 + (dy + 1) * 3 + k / 3;
                        v2 |= (uint32_t)__ldg(wsrc + tap * 256 + oc * 8 + k % 3) << (16 * hh);
                    }
                }
                h[jj] = v2;
            }
            reinterpret_cast<uint4*>(sw)[q * (TZ_WQ / 16) + kh * 48 + i * 16 + oc] = make_uint4(h[0], h[1], h[2], h[3]);
        }
    }
    for (int c = tid; c < TW_ZERO / 16; c += TZ_THREADS) reinterpret_cast<uint4*>(zt)[c] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t rb = smem_u32(sm), wb = smem_u32(sw);

    // bounded wait on barrier i for the phase of parity par, by one thread; false on a timeout
    // or once another role gave up
    auto wait_one = [&](int i, uint32_t par) -> bool {
        const uint32_t m = smem_u32(bar + i);
        for (int it = 0; it < (1 << 22); ++it) {
            if (tc_mbar_try(m, par)) return true;
            if (*(volatile int*)&abort_) return false;
        }
        atomicExch(&abort_, 1);
        return false;
    };
    // the same for a whole warp (lane 0 waits; the outcome is the warp's)
    auto wait_warp = [&](int i, uint32_t par) -> bool {
        int ok = 0;
        if (lane == 0) ok = wait_one(i, par);
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };
    double sq = 0.0;
    if (warp == 0) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const unsigned long long adesc0 = tc_desc(rb, TZ_PHALF, 128), bdesc0 = tc_desc(wb, TZ_WQ / 2, 128);
            const unsigned long long zdesc = tc_desc(smem_u32(zt), TW_ZERO / 2, 128);
            int issued = -1;
            for (int o = 0; o < zc; ++o) {
                bool ok = true;
                for (int i = o == 0 ? 0 : o + 2; i <= o + 2 && ok; ++i) ok = wait_one(FULL + i % TW_R, (i / TW_R) & 1);
                if (ok && o >= TW_S) ok = wait_one(SETE + o % TW_S, ((o / TW_S) - 1) & 1);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dset = tmem + (uint32_t)((o % TW_S) * 64);
                // the set's 4 rows cleared: zero A times any 64 rows of weights, not accumulated
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, 0, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(dset), "l"(zdesc), "l"(bdesc0), "r"(tc_idesc(64)) : "memory");
                unsigned long long abase[3];          // the plane's three input slots
#pragma unroll
                for (int dz = -1; dz <= 1; ++dz)
                    abase[dz + 1] = adesc0 + (unsigned long long)((((o + 1 + dz) % TW_R) * TZ_PLANE) / 16);
                // input rows outermost: the 9 MMAs of one row (dz, dx) share one accumulator range
#pragma unroll
                for (int ri = 0; ri < TZ_TY + 2; ++ri) {
                    const int b0 = ri - 2 > 0 ? ri - 2 : 0, b1 = ri < TZ_TY - 1 ? ri : TZ_TY - 1;
                    const int i0 = b0 - (ri - 2);          // first dy block fed (block i: dy = 1 - i)
                    const uint32_t idesc = tc_idesc((uint32_t)(16 * (b1 - b0 + 1)));
#pragma unroll
                    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
                        for (int dx = PACKX ? 0 : -1; dx <= (PACKX ? 0 : 1); ++dx) {
                            const int q = PACKX ? dz + 1 : (dz + 1) * 3 + dx + 1;
                            const unsigned long long ad = abase[dz + 1] + (unsigned long long)(ri * TZ_HX + dx + 1);
                            const unsigned long long bd =
                                bdesc0 + (unsigned long long)((q * TZ_WQ + i0 * 256) / 16);
                            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
                                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                         ::"r"(dset + 16 * b0), "l"(ad), "l"(bd), "r"(idesc) : "memory");
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(bar + SETF + o % TW_S)) : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(bar + EMPTY + o % TW_R)) : "memory");
                issued = o;
            }
            if (issued >= 0 && issued < zc - 1) {
                // stopped early: the MMAs in flight finish before tensor memory is released
                const uint32_t m = smem_u32(bar + SETF + issued % TW_S);
                for (int it = 0; it < (1 << 22) && !tc_mbar_try(m, (issued / TW_S) & 1); ++it) {}
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------------------------------------------------------- producers
        const int pt = tid - 32;
        uint32_t soff[TW_CPT], doff[TW_CPT];   // per copy: source (16-byte units, plane-relative), destination
#pragma unroll
        for (int k = 0; k < TW_CPT; ++k) {
            const int c = pt + TW_PROD * k;
            const int pp = c >> 1, h = c & 1;
            const int yy = pp / TZ_HX, xx = pp - yy * TZ_HX;
            const int gx = wrapc(x0 + xx - 1, a.nx), gy = wrapc(y0 + yy - 1, a.ny);
            soff[k] = (uint32_t)(((size_t)gy * a.nx + gx) * 2 + h);
            doff[k] = (uint32_t)(h * TZ_PHALF + pp * 16);
        }
        const size_t plane16 = (size_t)a.ny * a.nx * 2;
        bool ok = true;
        int i = 0;
        for (; i < zc + 2; ++i) {
            if (i >= TW_R && !wait_warp(EMPTY + i % TW_R, ((i / TW_R) - 1) & 1)) { ok = false; break; }
            const uint4* base = src + (size_t)wrapc(z0 - 1 + i, a.nz) * plane16;
            const uint32_t dst = rb + (uint32_t)((i % TW_R) * TZ_PLANE);
#pragma unroll
            for (int k = 0; k < TW_CPT; ++k)
                if (pt + TW_PROD * k < TZ_HY * TZ_HX * 2)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + doff[k]), "l"(base + soff[k])
                                 : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
            if (i >= TW_LAG) {   // input i - TW_LAG has landed: publish it to the MMA issuer
                asm volatile("cp.async.wait_group %0;" ::"n"(TW_LAG) : "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];"
                             ::"r"(smem_u32(bar + FULL + (i - TW_LAG) % TW_R)) : "memory");
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (ok) {   // the last TW_LAG inputs
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int j = zc + 2 - TW_LAG; j <= zc + 1; ++j)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar + FULL + j % TW_R))
                             : "memory");
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int wq = warp - 4;
        const int x = x0 + 32 * wq + lane;
        float bias[16];
        if (EPI == 0) {
#pragma unroll
            for (int n = 0; n < 16; ++n) bias[n] = __ldg(a.bias + n);
        }
        for (int o = 0; o < zc; ++o) {
            if (!wait_warp(SETF + o % TW_S, (o / TW_S) & 1)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tl = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)((o % TW_S) * 64);
            const long long pt0 = ((long long)(z0 + o) * a.ny + y0) * a.nx + x, rs = a.nx;   // row r: pt0 + r rs
            if (EPI == 0 || EPI == 3) {
                uint4 mk[TZ_TY][2];
                if (EPI == 3) {   // the rows' masks first, so that their loads overlap
#pragma unroll
                    for (int r = 0; r < TZ_TY; ++r) {
                        const uint4* mk4 = reinterpret_cast<const uint4*>(a.mask + (pt0 + r * rs) * 16);
                        mk[r][0] = __ldg(mk4);
                        mk[r][1] = __ldg(mk4 + 1);
                    }
                }
                uint32_t raw[TZ_TY][16];   // the set's 4 rows, loaded together, one wait
#pragma unroll
                for (int r = 0; r < TZ_TY; ++r) tc_ld16_async(tl + 16 * r, raw[r]);
#pragma unroll
                for (int r = 0; r < TZ_TY; ++r) tc_wait16(raw[r]);
#pragma unroll
                for (int r = 0; r < TZ_TY; ++r) {
                    float v[16];
#pragma unroll
                    for (int n = 0; n < 16; ++n) v[n] = __uint_as_float(raw[r][n]);
                    if (EPI == 0) {
#pragma unroll
                        for (int n = 0; n < 16; ++n) v[n] = fmaxf(v[n] + bias[n], 0.0f);
                    } else {
                        const uint32_t mw[8] = {mk[r][0].x, mk[r][0].y, mk[r][0].z, mk[r][0].w,
                                                mk[r][1].x, mk[r][1].y, mk[r][1].z, mk[r][1].w};
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            if (!(mw[q] & 0x7fffu)) v[2 * q] = 0.0f;
                            if (!(mw[q] & 0x7fff0000u)) v[2 * q + 1] = 0.0f;
                        }
                    }
                    uint32_t o2[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                        o2[q] = *reinterpret_cast<uint32_t*>(&h2);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(a.out + (pt0 + r * rs) * 16);
                    dst[0] = make_uint4(o2[0], o2[1], o2[2], o2[3]);
                    dst[1] = make_uint4(o2[4], o2[5], o2[6], o2[7]);
                }
            } else {
                double pn[TZ_TY], pm[TZ_TY], px[TZ_TY];   // the rows' pressures first (overlapped loads)
#pragma unroll
                for (int r = 0; r < TZ_TY; ++r) {
                    pn[r] = a.pn[pt0 + r * rs];
                    pm[r] = a.pnm1[pt0 + r * rs];
                    px[r] = EPI == 2 ? a.pnext[pt0 + r * rs] : 0.0;
                }
                const float b0 = __ldg(a.bias);
                uint32_t raw[TZ_TY];
#pragma unroll
                for (int r = 0; r < TZ_TY; ++r) raw[r] = tc_ld1_async(tl + 16 * r);
                tc_wait4(raw);
#pragma unroll
                for (int r = 0; r < TZ_TY; ++r) {
                    const double y = (double)(__uint_as_float(raw[r]) + b0);
                    if (EPI == 1) {
                        a.phat[pt0 + r * rs] = 2.0 * pn[r] - pm[r] + a.sc[0] * y;
                    } else {
                        const double e = y - (px[r] - (2.0 * pn[r] - pm[r])) * a.sc[1];
                        sq += e * e;
                        a.out[(pt0 + r * rs) * 16] = __double2bfloat16(a.gscale * e);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar + SETE + o % TW_S))
                                        : "memory");
        }
        if (EPI == 2) {
            for (int s2 = 16; s2 > 0; s2 >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s2);
            if (lane == 0) ws[wq] = sq;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
        if (abort_) atomicExch(a.err, 1);
        if (EPI == 2) a.red[blockIdx.x] = ws[0] + ws[1] + ws[2] + ws[3];
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TZ_TMEM_COLS) : "memory");
}

// tcgen05 convolution for nx = 64 (the 64^3 training windows): a CTA owns one pair of y rows
// (M = 128 = 2 rows x 64 points: TMEM lane i is row i / 64, x = i % 64) and marches zc planes
// like k_pnet_conv_tcz.  An MMA's A operand must be 16 core matrices of 8 points at one stride,
// so each input plane (rows y0-1 .. y0+2, both 8-channel halves) is stored three times, row by
// row rotated by dx = -1, 0, +1 (copy v holds in[(x + v - 1) mod 64] at x): the window of tap
// (dz, dy, dx) is rows dy+1 and dy+2 of copy dx+1, 128 consecutive 16-byte points.  One thread
// issues the 27 MMAs of an output plane; warps 0-3 run the epilogue.
constexpr int T64_ROWS = 4;                              // input rows of a plane (2 + halo)
constexpr int T64_HALF = T64_ROWS * 64 * 16;             // one 8-channel half of one copy (4096 B)
constexpr int T64_COPY = 2 * T64_HALF;                   // 8192 B
constexpr int T64_PLANE = 3 * T64_COPY;                  // 24576 B
constexpr int T64_SMEM = 4 * T64_PLANE + 27 * 512 + 32;  // ring + weights + 2 mbarriers + TMEM slot
constexpr int T64_TMEM_COLS = 32;                        // 2 sets x 16 columns

__device__ __forceinline__ void t64_load_plane(const uint4* __restrict__ src, unsigned char* dstp, int y0, int gz,
                                               int ny) {
    constexpr int NC = T64_ROWS * 64 * 2, BT = 2;        // 512 16-byte pieces, 2 per thread
    uint4 v[BT];
    int yy[BT], xg[BT], h[BT];
#pragma unroll
    for (int q = 0; q < BT; ++q) {
        const int c = threadIdx.x + q * TZ_THREADS;
        h[q] = c & 1;
        const int pp = c >> 1;
        yy[q] = pp >> 6;
        xg[q] = pp & 63;
        const int gy = wrapc(y0 + yy[q] - 1, ny);
        const long long pt = ((long long)gz * ny + gy) * 64 + xg[q];
        v[q] = __ldg(src + pt * 2 + h[q]);
    }
    static_assert(NC == BT * TZ_THREADS, "one pass");
#pragma unroll
    for (int q = 0; q < BT; ++q) {
#pragma unroll
        for (int cv = 0; cv < 3; ++cv) {                 // copy cv holds in[x + cv - 1] at x
            const int xd = (xg[q] - (cv - 1)) & 63;
            *reinterpret_cast<uint4*>(dstp + cv * T64_COPY + h[q] * T64_HALF + (yy[q] * 64 + xd) * 16) = v[q];
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(TZ_THREADS, 2) k_pnet_conv_tcz64(ConvArgs a, int zc) {
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* ring = sm;
    unsigned char* sw = sm + 4 * T64_PLANE;
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sw + 27 * 512);   // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sw + 27 * 512 + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npair = a.ny / 2;
    const int b = blockIdx.x;
    const int y0 = (b % npair) * 2, z0 = (b / npair) * zc;
    const uint4* src = reinterpret_cast<const uint4*>(a.in);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(T64_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {   // one commit per output plane
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar + 1)), "r"(1) : "memory");
    }
    {
        const uint4* wsrc = reinterpret_cast<const uint4*>(a.wtc);
        for (int c = tid; c < 27 * 32; c += TZ_THREADS) reinterpret_cast<uint4*>(sw)[c] = __ldg(wsrc + c);
    }
    for (int lp = 0; lp < 3; ++lp) t64_load_plane(src, ring + lp * T64_PLANE, y0, wrapc(z0 - 1 + lp, a.nz), a.ny);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t rb = smem_u32(ring), wb = smem_u32(sw);
    const int wq = warp & 3;                              // tensor-memory lane quadrant of this warp
    const int orow = wq >> 1, x = 32 * (wq & 1) + lane;   // lane 32 wq + lane: row (32 wq + lane) / 64
    float bias[16];
    if (EPI == 0) {
#pragma unroll
        for (int n = 0; n < 16; ++n) bias[n] = __ldg(a.bias + n);
    }
    uint32_t ph0 = 0u, ph1 = 0u;
    bool fail = false;
    double sq = 0.0;
    auto epilogue = [&](int o) {                          // output plane o (accumulator set o & 1)
        if (warp >= 4) return;
        const uint32_t tl = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)((o & 1) * 16);
        const int z = z0 + o;
        const long long pt = ((long long)z * a.ny + (y0 + orow)) * 64 + x;
        if (EPI == 0 || EPI == 3) {
            float v[16];
            tc_ld16(tl, v);
            if (EPI == 0) {
#pragma unroll
                for (int n = 0; n < 16; ++n) v[n] = fmaxf(v[n] + bias[n], 0.0f);
            } else {
                const uint4* mk4 = reinterpret_cast<const uint4*>(a.mask + pt * 16);
                const uint4 m0 = __ldg(mk4), m1 = __ldg(mk4 + 1);
                const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (!(mw[q] & 0x7fffu)) v[2 * q] = 0.0f;
                    if (!(mw[q] & 0x7fff0000u)) v[2 * q + 1] = 0.0f;
                }
            }
            uint32_t o2[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                o2[q] = *reinterpret_cast<uint32_t*>(&h2);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.out + pt * 16);
            dst[0] = make_uint4(o2[0], o2[1], o2[2], o2[3]);
            dst[1] = make_uint4(o2[4], o2[5], o2[6], o2[7]);
        } else {
            const double y = (double)(tc_ld1(tl) + __ldg(a.bias));
            const double pn = a.pn[pt], pm = a.pnm1[pt];
            if (EPI == 1) {
                a.phat[pt] = 2.0 * pn - pm + a.sc[0] * y;
            } else {
                const double e = y - (a.pnext[pt] - (2.0 * pn - pm)) * a.sc[1];
                sq += e * e;
                a.out[pt * 16] = __double2bfloat16(a.gscale * e);
            }
        }
    };
    auto wait_set = [&](int o) -> bool {                  // MMAs of output plane o are complete (bounded)
        const uint32_t m = smem_u32(mbar + (o & 1));
        const uint32_t par = (o & 1) ? ph1 : ph0;
        bool done = false;
        for (int i = 0; i < (1 << 22) && !done; ++i) done = tc_mbar_try(m, par);
        if (o & 1) ph1 ^= 1u; else ph0 ^= 1u;
        const bool ok = __syncthreads_and(done);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return ok;
    };
    // A: ring slot, copy dx + 1, first row dy + 1 (64 points of 16 bytes a row); both K halves
    // one half apart (leading byte offset), core matrices of 8 points 128 bytes apart
    const unsigned long long adesc0 = tc_desc(rb, T64_HALF, 128), bdesc0 = tc_desc(wb, 256, 128);
    for (int o = 0; o < zc; ++o) {
        if (tid == 0) {
            const uint32_t dcol = tmem + (uint32_t)((o & 1) * 16);
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                const int slot = (o + 1 + dz) & 3;
                const unsigned long long ad = adesc0 + (unsigned long long)((slot * T64_PLANE + (dx + 1) * T64_COPY) / 16 +
                                                                              (dy + 1) * 64);
                const unsigned long long bd = bdesc0 + (unsigned long long)(tap * 32);
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(dcol), "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(tap) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(mbar + (o & 1))) : "memory");
        }
        __syncwarp();
        if (o > 0) {
            // plane o-1 is done: store it; its last input plane's slot is free for input plane o+3
            if (wait_set(o - 1)) epilogue(o - 1);
            else fail = true;
        }
        if (o + 3 <= zc + 1) t64_load_plane(src, ring + ((o + 3) & 3) * T64_PLANE, y0, wrapc(z0 + o + 2, a.nz), a.ny);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (wait_set(zc - 1)) epilogue(zc - 1);
    else fail = true;
    if (fail && tid == 0) atomicExch(a.err, 1);
    if (EPI == 2) {
        __shared__ double ws[TZ_THREADS / 32];
        for (int s2 = 16; s2 > 0; s2 >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s2);
        if (lane == 0) ws[warp] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < TZ_THREADS / 32; ++w) t += ws[w];
            a.red[blockIdx.x] = t;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T64_TMEM_COLS) : "memory");
}

// Weight gradient of one layer over the CTA's tile:
//   part[cta][tap][o][i] = sum_v dz(v)[o] act(v + tap)[i],  part[cta][6912 + o] = sum_v dz(v)[o]
__global__ void __launch_bounds__(THREADS, 2) k_pnet_wgrad(const __nv_bfloat16* __restrict__ dz,
                                                           const __nv_bfloat16* __restrict__ act,
                                                           float* __restrict__ part, int nx, int ny, int nz) {
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* sin = sm;
    unsigned char* sdz = sm + SMEM_IN;
    const TileOrigin o = tile_origin(nx, ny);
    load_halo(act, sin, o, nx, ny, nz);
    {
        const uint4* src = reinterpret_cast<const uint4*>(dz);
        for (int c = threadIdx.x; c < TILE_PTS * 2; c += THREADS) {
            const int q = c >> 1, h = c & 1;
            const int xl = q % TX, yl = (q / TX) % TY, zl = q / (TX * TY);
            const long long pt = ((long long)(o.z0 + zl) * ny + (o.y0 + yl)) * nx + o.x0 + xl;
            *reinterpret_cast<uint4*>(sdz + swz(q, h)) = __ldg(src + pt * 2 + h);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntap = warp < 3 ? 4 : 3;                 // taps warp, warp + 8, warp + 16 (, warp + 24)
    const uint32_t sin_u = smem_u32(sin), sdz_u = smem_u32(sdz);
    const int r = lane & 7, j = lane >> 3;
    float acc[4][2][4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[s][nt][q] = 0.0f;
#pragma unroll 1
    for (int chunk = 0; chunk < TILE_PTS / 16; ++chunk) {
        const int zl = chunk >> 4, yl = (chunk >> 1) & 7, xh = chunk & 1;
        uint32_t av[4];
        {
            const int q = (zl * TY + yl) * TX + xh * 16 + r + 8 * (j >> 1);
            ldsm_x4_t(sdz_u + swz(q, j & 1), av);
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (s < ntap) {
                const int tap = warp + 8 * s;
                const int dzz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                const int sp = ((zl + dzz + 1) * HY + (yl + dy + 1)) * HX + xh * 16 + dx + 1 + r + 8 * (j & 1);
                uint32_t bv[4];
                ldsm_x4_t(sin_u + swz(sp, j >> 1), bv);
                mma_bf16(acc[s][0], av, bv[0], bv[1]);
                mma_bf16(acc[s][1], av, bv[2], bv[3]);
            }
        }
    }
    float* dst = part + (size_t)blockIdx.x * PN_PART;
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (s < ntap) {
            const int tap = warp + 8 * s;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int i = nt * 8 + 2 * t4;
                *reinterpret_cast<float2*>(dst + tap * 256 + g * 16 + i) = make_float2(acc[s][nt][0], acc[s][nt][1]);
                *reinterpret_cast<float2*>(dst + tap * 256 + (g + 8) * 16 + i) = make_float2(acc[s][nt][2], acc[s][nt][3]);
            }
        }
    }
    // bias gradient: channel oc = tid & 15 summed over points q = tid >> 4 (mod 16)
    __shared__ float bs[THREADS];
    {
        const int oc = threadIdx.x & 15, q0 = threadIdx.x >> 4;
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(sdz);
        float s = 0.0f;
        for (int q = q0; q < TILE_PTS; q += 16) s += __bfloat162float(e[swz(q, oc >> 3) / 2 + (oc & 7)]);
        bs[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        float s = 0.0f;
        for (int q = 0; q < 16; ++q) s += bs[q * 16 + threadIdx.x];
        dst[6912 + threadIdx.x] = s;
    }
}

// grad[param] = sum over CTAs of the partials (fixed order, FP64 accumulation).
__global__ void k_pnet_reduce(const float* __restrict__ part, int ncta, float* __restrict__ grad) {
    const int l = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= PN_PART) return;
    int pidx;
    if (e < 6912) {
        const int tap = e >> 8, oc = (e >> 4) & 15, ic = e & 15;
        if (oc >= lay_out(l) || ic >= lay_in(l)) return;
        pidx = lay_w(l) + (oc * lay_in(l) + ic) * 27 + tap;
    } else {
        const int oc = e - 6912;
        if (oc >= lay_out(l)) return;
        pidx = lay_b(l) + oc;
    }
    const float* p = part + (size_t)l * ncta * PN_PART + e;
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += p[(size_t)c * PN_PART];
    grad[pidx] = (float)s;
}

// Adam step (optional) and packing of the bfloat16 weights.
__global__ void k_pnet_adam_pack(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                                 const float* __restrict__ grad, int adam, float lr, float bc1, float bc2,
                                 __nv_bfloat16* __restrict__ wf, __nv_bfloat16* __restrict__ wb,
                                 __nv_bfloat16* __restrict__ wtf, __nv_bfloat16* __restrict__ wtb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= PN_NP) return;
    float x = w[p];
    if (adam) {
        const float gr = grad[p];
        const float mm = 0.9f * m[p] + 0.1f * gr;
        const float vv = 0.999f * v[p] + 0.001f * gr * gr;
        m[p] = mm;
        v[p] = vv;
        x -= lr * (mm * bc1) / (sqrtf(vv * bc2) + 1e-8f);
        w[p] = x;
    }
    int l = 0;
    while (l < 3 && p >= lay_w(l + 1)) ++l;
    if (p >= lay_b(l)) return;                   // a bias: used in FP32
    const int q = p - lay_w(l);
    const int tap = q % 27, ic = (q / 27) % lay_in(l), oc = q / (27 * lay_in(l));
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    wf[(size_t)l * PN_WPK + (tap * 16 + oc) * 24 + ic] = h;
    if (l > 0) wb[(size_t)l * PN_WPK + ((26 - tap) * 16 + ic) * 24 + oc] = h;
    // tcgen05 layout [tap][K half][row n][8 k]: forward rows = output channels, k = inputs;
    // backward-data rows = input channels, k = output channels, taps reversed
    wtf[(size_t)l * PN_TCW + tap * 256 + (ic >> 3) * 128 + oc * 8 + (ic & 7)] = h;
    if (l > 0) wtb[(size_t)l * PN_TCW + (26 - tap) * 256 + (oc >> 3) * 128 + ic * 8 + (oc & 7)] = h;
}

__global__ void k_pnet_sumsq(const double* __restrict__ x, long long n, double* __restrict__ red) {
    double s = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        s += x[c] * x[c];
    __shared__ double ws[THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) t += ws[w];
        red[blockIdx.x] = t;
    }
}

// what 0: sc[0] = s = sqrt(S / n) (1 if 0), sc[1] = 1/s;  what 1: sc[2] = S / n (loss)
__global__ void k_pnet_fin(const double* __restrict__ red, int nblk, double* __restrict__ sc, int what, double inv_n) {
    __shared__ double ws[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += red[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        if (what == 0) {
            double sv = sqrt(t * inv_n);
            if (!(sv > 0.0)) sv = 1.0;
            sc[0] = sv;
            sc[1] = 1.0 / sv;
        } else {
            sc[2] = t * inv_n;
        }
    }
}

// Features of point c as bfloat16 bits (the rounding of the 3-channel input layout).
__device__ __forceinline__ void pn_feat_bits(const double* __restrict__ rho, double rho0, const double* __restrict__ pn,
                                             const double* __restrict__ pnm1, double is, long long c, uint32_t (&b)[3]) {
    const __nv_bfloat16 h0 = __double2bfloat16(1.0 - rho0 / rho[c]);
    const __nv_bfloat16 h1 = __double2bfloat16(pn[c] * is);
    const __nv_bfloat16 h2 = __double2bfloat16(pnm1[c] * is);
    b[0] = *reinterpret_cast<const unsigned short*>(&h0);
    b[1] = *reinterpret_cast<const unsigned short*>(&h1);
    b[2] = *reinterpret_cast<const unsigned short*>(&h2);
}

// feat: the 3 features of each point in channels 0-2 of its 16 (the others stay zero).
__global__ void k_pnet_features(const double* __restrict__ rho, double rho0, const double* __restrict__ pn,
                                const double* __restrict__ pnm1, const double* __restrict__ sc, long long n,
                                __nv_bfloat16* __restrict__ feat) {
    const double is = sc[1];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        uint32_t m[3];
        pn_feat_bits(rho, rho0, pn, pnm1, is, c, m);
        *reinterpret_cast<uint2*>(feat + c * 16) = make_uint2(m[0] | (m[1] << 16), m[2]);
    }
}

// The same with the tcgen05 first layer's input: one CTA of nx threads per x row (nx <= 1024),
// each point's features computed once and shared through shared memory; featx holds at channel
// 3 (dx + 1) + c the feature c of the point x + dx (periodic in x), channels 9-15 zero.
__global__ void k_pnet_features_x(const double* __restrict__ rho, double rho0, const double* __restrict__ pn,
                                  const double* __restrict__ pnm1, const double* __restrict__ sc,
                                  __nv_bfloat16* __restrict__ feat, __nv_bfloat16* __restrict__ featx) {
    __shared__ uint2 row[1024];
    const int nx = blockDim.x, ix = threadIdx.x;
    const long long c = (long long)blockIdx.x * nx + ix;
    uint32_t m[3];
    pn_feat_bits(rho, rho0, pn, pnm1, sc[1], c, m);
    const uint2 u = make_uint2(m[0] | (m[1] << 16), m[2]);
    *reinterpret_cast<uint2*>(feat + c * 16) = u;
    row[ix] = u;
    __syncthreads();
    const uint2 w = row[ix == 0 ? nx - 1 : ix - 1], e = row[ix == nx - 1 ? 0 : ix + 1];
    // bf16 lanes: u.x = (f0, f1), u.y = (f2, 0), likewise w and e
    uint4* dst = reinterpret_cast<uint4*>(featx + c * 16);
    dst[0] = make_uint4(w.x, (w.y & 0xffffu) | (u.x << 16), (u.x >> 16) | (u.y << 16), e.x);
    dst[1] = make_uint4(e.y & 0xffffu, 0u, 0u, 0u);
}

}  // namespace

struct flups_pnet_s {
    int nx, ny, nz, dev, ncta, nred;
    long long n;
    cudaStream_t stream;
    float* w; float* m; float* v; float* grad;    // FP32 master weights, Adam moments, gradient
    __nv_bfloat16* wf; __nv_bfloat16* wb;         // packed bfloat16 weights (4 layers each)
    __nv_bfloat16* wtf; __nv_bfloat16* wtb;       // the same in the tcgen05 layout
    int* err;                                     // device error word (bounded waits)
    int use_tc;                                   // tcgen05 convolutions: 2 nx % 128 == 0, nx <= 1024 (all), 1 nx == 64 (output layer)
    int last_red;                                 // CTAs of the last loss partials
    __nv_bfloat16* feat; __nv_bfloat16* act[3]; __nv_bfloat16* dy; __nv_bfloat16* g[2];
    float* part;                                  // weight-gradient partials [4][ncta][PN_PART]
    double* red;                                  // per-CTA scalar partials
    double* sc;                                   // s, 1/s, loss
    double* sc_host;
    void* base;
    int step;
    unsigned long long launches;
    // optional per-kernel timing (flups_pnet_set_profiling)
    int prof_on, prof_n, prof_cap, prof_open;
    cudaEvent_t* prof_ev;
    int* prof_kid;
    double prof_ms[FLUPS_PNET_NKERNELS];
    long long prof_cnt[FLUPS_PNET_NKERNELS];
};

static const char* kPnetKernelNames[FLUPS_PNET_NKERNELS] = {
    "k_pnet_features", "k_pnet_conv_hidden", "k_pnet_conv_out", "k_pnet_conv_bwd", "k_pnet_wgrad", "k_pnet_update"};

namespace {

enum { PK_FEATURES = 0, PK_CONV_HIDDEN, PK_CONV_OUT, PK_CONV_BWD, PK_WGRAD, PK_UPDATE };

void pk_begin(flups_pnet N, int kid) {
    N->prof_open = 0;
    if (!N->prof_on || N->prof_n >= N->prof_cap) return;
    if (cudaEventRecord(N->prof_ev[2 * N->prof_n], N->stream) != cudaSuccess) return;
    N->prof_kid[N->prof_n] = kid;
    N->prof_open = 1;
}

void pk_end(flups_pnet N) {
    if (!N->prof_open) return;
    N->prof_open = 0;
    if (cudaEventRecord(N->prof_ev[2 * N->prof_n + 1], N->stream) == cudaSuccess) N->prof_n++;
}

struct PnGuard {
    int prev = -1;
    explicit PnGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~PnGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

flups_status pn_status(cudaError_t e) {
    if (e == cudaSuccess) return FLUPS_OK;
    flups_note_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? FLUPS_ENOMEM : FLUPS_ECUDA;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t set_smem_attrs() {
    static int done = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_pnet_conv<2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv<2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, WGRAD_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv_tcz<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TZ_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv_tcz<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TZ_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv_tcz<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TZ_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv_tcz<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TZ_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv_tcz<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TZ_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv_tcz64<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, T64_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pnet_conv_tcz64<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, T64_SMEM);
    if (e == cudaSuccess) done = dev;
    return e;
}

ConvArgs conv_args(flups_pnet N) {
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.sc = N->sc;
    a.red = N->red;
    a.err = N->err;
    a.nx = N->nx; a.ny = N->ny; a.nz = N->nz;
    return a;
}

// first: the layer reads the 3-channel features; on the tcgen05 path it reads them with their x
// neighbours packed (N->g[0], written by k_pnet_features) and takes the three x taps in K
template <int NT, int EPI>
void conv(flups_pnet N, const ConvArgs& a, bool first = false) {
    pk_begin(N, EPI == 0 ? PK_CONV_HIDDEN : (EPI == 3 ? PK_CONV_BWD : PK_CONV_OUT));
    if (N->use_tc == 2) {
        const int zc = N->nz % 16 == 0 ? 16 : (N->nz % 8 == 0 ? 8 : 4);
        const int nb = (N->nx / 128) * (N->ny / TZ_TY) * (N->nz / zc);
        if (EPI == 0 && first) {
            ConvArgs b = a;
            b.in = N->g[0];
            k_pnet_conv_tcz<0, true><<<nb, TZ_THREADS, TZ_SMEM, N->stream>>>(b, zc);
        } else {
            k_pnet_conv_tcz<EPI, false><<<nb, TZ_THREADS, TZ_SMEM, N->stream>>>(a, zc);
        }
        if (EPI == 2) N->last_red = nb;
    } else if (N->use_tc == 1 && (EPI == 1 || EPI == 2)) {
        // nx = 64: the row-pair tcgen05 kernel for the 16 -> 1 output layer (measured 20 % faster
        // than mma.sync at 64^3); the 16-channel layers stay on mma.sync (17 % faster there: the
        // row-pair kernel stores each input point three times for 128 outputs a plane)
        const int zc = N->nz % 8 == 0 ? 8 : 4;
        const int nb = (N->ny / 2) * (N->nz / zc);
        k_pnet_conv_tcz64<EPI><<<nb, TZ_THREADS, T64_SMEM, N->stream>>>(a, zc);
        if (EPI == 2) N->last_red = nb;
    } else {
        k_pnet_conv<NT, EPI><<<N->ncta, THREADS, CONV_SMEM, N->stream>>>(a);
        if (EPI == 2) N->last_red = N->ncta;
    }
    pk_end(N);
    N->launches++;
}

void pack(flups_pnet N, int adam, float lr) {
    float bc1 = 1.0f, bc2 = 1.0f;
    if (adam) {
        N->step++;
        bc1 = (float)(1.0 / (1.0 - std::pow(0.9, N->step)));
        bc2 = (float)(1.0 / (1.0 - std::pow(0.999, N->step)));
    }
    pk_begin(N, PK_UPDATE);
    k_pnet_adam_pack<<<(PN_NP + 255) / 256, 256, 0, N->stream>>>(N->w, N->m, N->v, N->grad, adam, lr, bc1, bc2, N->wf,
                                                                 N->wb, N->wtf, N->wtb);
    pk_end(N);
    N->launches++;
}

// features + layers 1..3 (hidden activations)
void forward_hidden(flups_pnet N, const double* rho, double rho0, const double* pn, const double* pnm1) {
    cudaStream_t s = N->stream;
    pk_begin(N, PK_FEATURES);
    k_pnet_sumsq<<<N->nred, THREADS, 0, s>>>(pn, N->n, N->red);
    k_pnet_fin<<<1, 1024, 0, s>>>(N->red, N->nred, N->sc, 0, 1.0 / (double)N->n);
    // the tcgen05 first layer reads its x-tap-packed input from N->g[0] (free in the forward pass)
    if (N->use_tc == 2)
        k_pnet_features_x<<<(unsigned)(N->n / N->nx), N->nx, 0, s>>>(rho, rho0, pn, pnm1, N->sc, N->feat, N->g[0]);
    else
        k_pnet_features<<<N->nred, THREADS, 0, s>>>(rho, rho0, pn, pnm1, N->sc, N->n, N->feat);
    pk_end(N);
    N->launches += 3;
    const __nv_bfloat16* in = N->feat;
    for (int l = 0; l < 3; ++l) {
        ConvArgs a = conv_args(N);
        a.in = in;
        a.w = N->wf + (size_t)l * PN_WPK;
        a.wtc = N->wtf + (size_t)l * PN_TCW;
        a.bias = N->w + lay_b(l);
        a.out = N->act[l];
        conv<2, 0>(N, a, l == 0);
        in = N->act[l];
    }
}

void wgrad(flups_pnet N, int l, const __nv_bfloat16* dz, const __nv_bfloat16* act) {
    pk_begin(N, PK_WGRAD);
    k_pnet_wgrad<<<N->ncta, THREADS, WGRAD_SMEM, N->stream>>>(dz, act, N->part + (size_t)l * N->ncta * PN_PART, N->nx,
                                                              N->ny, N->nz);
    pk_end(N);
    N->launches++;
}

// Reads (and clears) the device error word: FLUPS_ETIMEOUT if a bounded wait gave up.  Synchronises.
flups_status check_err(flups_pnet N) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, N->err, sizeof(int), cudaMemcpyDeviceToHost, N->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(N->stream);
    if (e != cudaSuccess) return pn_status(e);
    if (h) {
        cudaMemsetAsync(N->err, 0, sizeof(int), N->stream);
        return FLUPS_ETIMEOUT;
    }
    return FLUPS_OK;
}

flups_status check_fields(flups_pnet N, const double* rho, double rho0, const double* pn, const double* pnm1) {
    if (!N || !rho || !pn || !pnm1) return FLUPS_EINVAL;
    if (!al16(rho) || !al16(pn) || !al16(pnm1)) return FLUPS_EINVAL;
    if (!(rho0 > 0.0) || !std::isfinite(rho0)) return FLUPS_EINVAL;
    return FLUPS_OK;
}

}  // namespace

extern "C" {

flups_status flups_pnet_create(flups_pnet* out, int nx, int ny, int nz, const float* params, void* stream) {
    if (!out) return FLUPS_EINVAL;
    *out = nullptr;
    if (!params) return FLUPS_EINVAL;
    if (nx < TX || ny < TY || nz < TZ) return FLUPS_EUNSUPPORTED;
    if (nx % TX || ny % TY || nz % TZ) return FLUPS_EUNSUPPORTED;
    if ((long long)nx * ny * nz > (1LL << 28)) return FLUPS_EUNSUPPORTED;
    for (int p = 0; p < PN_NP; ++p)
        if (!std::isfinite(params[p])) return FLUPS_EINVAL;
    flups_pnet N = new (std::nothrow) flups_pnet_s();
    if (!N) return FLUPS_ENOMEM;
    N->nx = nx; N->ny = ny; N->nz = nz;
    N->n = (long long)nx * ny * nz;
    N->ncta = (int)(N->n / TILE_PTS);
    N->nred = (int)std::min<long long>((N->n + 4 * THREADS - 1) / (4 * THREADS), 1216);
    N->stream = (cudaStream_t)stream;
    cudaGetDevice(&N->dev);
    cudaError_t e = set_smem_attrs();
    if (e != cudaSuccess) { delete N; return pn_status(e); }
    const size_t fbytes = (size_t)N->n * 16 * sizeof(__nv_bfloat16);
    const size_t off_w = 0, off_wf = 4 * (size_t)16384 * 4;
    const size_t off_wb = off_wf + 4 * (size_t)PN_WPK * 2;
    const size_t off_wtf = off_wb + 4 * (size_t)PN_WPK * 2;
    const size_t off_wtb = off_wtf + 4 * (size_t)PN_TCW * 2;
    const size_t off_err = off_wtb + 4 * (size_t)PN_TCW * 2;
    const size_t off_feat = (off_err + 16 + 255) / 256 * 256;
    const size_t off_part = off_feat + 7 * fbytes;
    const size_t off_red = off_part + 4 * (size_t)N->ncta * PN_PART * sizeof(float);
    const size_t off_sc = off_red + (size_t)std::max(N->nred, 2 * N->ncta) * sizeof(double);
    const size_t total = off_sc + 8 * sizeof(double);
    e = cudaMalloc(&N->base, total);
    if (e != cudaSuccess) { delete N; return pn_status(e); }
    unsigned char* b = (unsigned char*)N->base;
    N->w = (float*)(b + off_w);
    N->m = N->w + 16384;
    N->v = N->m + 16384;
    N->grad = N->v + 16384;
    N->wf = (__nv_bfloat16*)(b + off_wf);
    N->wb = (__nv_bfloat16*)(b + off_wb);
    N->wtf = (__nv_bfloat16*)(b + off_wtf);
    N->wtb = (__nv_bfloat16*)(b + off_wtb);
    N->err = (int*)(b + off_err);
    N->use_tc = nx % 128 == 0 && nx <= 1024 ? 2 : (nx == 64 ? 1 : 0);
    N->last_red = N->ncta;
    __nv_bfloat16* f = (__nv_bfloat16*)(b + off_feat);
    const size_t fe = (size_t)N->n * 16;
    N->feat = f;
    N->act[0] = f + fe; N->act[1] = f + 2 * fe; N->act[2] = f + 3 * fe;
    N->dy = f + 4 * fe; N->g[0] = f + 5 * fe; N->g[1] = f + 6 * fe;
    N->part = (float*)(b + off_part);
    N->red = (double*)(b + off_red);
    N->sc = (double*)(b + off_sc);
    e = cudaMallocHost(&N->sc_host, 8 * sizeof(double));
    if (e != cudaSuccess) { cudaFree(N->base); delete N; return pn_status(e); }
    // zero: moments, packed weights (padding), feature and output-gradient channels never written
    e = cudaMemsetAsync(b, 0, off_feat, N->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(N->feat, 0, fbytes, N->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(N->dy, 0, fbytes, N->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(N->w, params, PN_NP * sizeof(float), cudaMemcpyHostToDevice, N->stream);
    if (e == cudaSuccess) { pack(N, 0, 0.0f); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = cudaStreamSynchronize(N->stream);
    if (e != cudaSuccess) {
        cudaFreeHost(N->sc_host);
        cudaFree(N->base);
        delete N;
        return pn_status(e);
    }
    *out = N;
    return FLUPS_OK;
}

flups_status flups_pnet_destroy(flups_pnet N) {
    if (!N) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    cudaError_t e = cudaStreamSynchronize(N->stream);
    cudaFree(N->base);
    cudaFreeHost(N->sc_host);
    if (N->prof_ev) {
        for (int q = 0; q < 2 * N->prof_cap; ++q) cudaEventDestroy(N->prof_ev[q]);
        std::free(N->prof_ev);
        std::free(N->prof_kid);
    }
    delete N;
    return pn_status(e);
}

flups_status flups_pnet_set_profiling(flups_pnet N, int on) {
    if (!N) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    if (on && !N->prof_ev) {
        const int cap = 1024;
        N->prof_ev = (cudaEvent_t*)std::calloc(2 * cap, sizeof(cudaEvent_t));
        N->prof_kid = (int*)std::calloc(cap, sizeof(int));
        if (!N->prof_ev || !N->prof_kid) return FLUPS_ENOMEM;
        for (int q = 0; q < 2 * cap; ++q)
            if (cudaEventCreate(&N->prof_ev[q]) != cudaSuccess) return FLUPS_ECUDA;
        N->prof_cap = cap;
    }
    N->prof_on = on ? 1 : 0;
    N->prof_n = 0;
    for (int q = 0; q < FLUPS_PNET_NKERNELS; ++q) { N->prof_ms[q] = 0.0; N->prof_cnt[q] = 0; }
    return FLUPS_OK;
}

flups_status flups_pnet_profile_read(flups_pnet N, double* ms, long long* n) {
    if (!N || !ms || !n) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    cudaError_t e = cudaStreamSynchronize(N->stream);
    if (e != cudaSuccess) return pn_status(e);
    for (int q = 0; q < N->prof_n; ++q) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, N->prof_ev[2 * q], N->prof_ev[2 * q + 1]) == cudaSuccess) {
            N->prof_ms[N->prof_kid[q]] += t;
            N->prof_cnt[N->prof_kid[q]] += 1;
        }
    }
    N->prof_n = 0;
    for (int q = 0; q < FLUPS_PNET_NKERNELS; ++q) {
        ms[q] = N->prof_ms[q];
        n[q] = N->prof_cnt[q];
        N->prof_ms[q] = 0.0;
        N->prof_cnt[q] = 0;
    }
    return FLUPS_OK;
}

const char* flups_pnet_kernel_name(int id) {
    return (id >= 0 && id < FLUPS_PNET_NKERNELS) ? kPnetKernelNames[id] : "unknown";
}

flups_status flups_pnet_set_params(flups_pnet N, const float* params) {
    if (!N || !params) return FLUPS_EINVAL;
    for (int p = 0; p < PN_NP; ++p)
        if (!std::isfinite(params[p])) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    cudaError_t e = cudaMemcpyAsync(N->w, params, PN_NP * sizeof(float), cudaMemcpyHostToDevice, N->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(N->m, 0, 2 * 16384 * sizeof(float), N->stream);
    if (e == cudaSuccess) { pack(N, 0, 0.0f); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = cudaStreamSynchronize(N->stream);   // params may be freed on return
    N->step = 0;
    return pn_status(e);
}

flups_status flups_pnet_get_params(flups_pnet N, float* params) {
    if (!N || !params) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    cudaError_t e = cudaMemcpyAsync(params, N->w, PN_NP * sizeof(float), cudaMemcpyDeviceToHost, N->stream);
    if (e != cudaSuccess) return pn_status(e);
    return check_err(N);
}

flups_status flups_pnet_get_adam(flups_pnet N, float* m, float* v, long long* step) {
    if (!N || !m || !v || !step) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    cudaError_t e = cudaMemcpyAsync(m, N->m, PN_NP * sizeof(float), cudaMemcpyDeviceToHost, N->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, N->v, PN_NP * sizeof(float), cudaMemcpyDeviceToHost, N->stream);
    if (e != cudaSuccess) return pn_status(e);
    *step = N->step;
    return check_err(N);
}

flups_status flups_pnet_set_adam(flups_pnet N, const float* m, const float* v, long long step) {
    if (!N || !m || !v || step < 0 || step > 0x7FFFFFFFLL) return FLUPS_EINVAL;
    for (int p = 0; p < PN_NP; ++p)
        if (!std::isfinite(m[p]) || !std::isfinite(v[p]) || v[p] < 0.0f) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    cudaError_t e = cudaMemcpyAsync(N->m, m, PN_NP * sizeof(float), cudaMemcpyHostToDevice, N->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(N->v, v, PN_NP * sizeof(float), cudaMemcpyHostToDevice, N->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(N->stream);   // m, v may be freed on return
    if (e == cudaSuccess) N->step = (int)step;
    return pn_status(e);
}

flups_status flups_pnet_get_grads(flups_pnet N, float* grads) {
    if (!N || !grads) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    cudaError_t e = cudaMemcpyAsync(grads, N->grad, PN_NP * sizeof(float), cudaMemcpyDeviceToHost, N->stream);
    if (e != cudaSuccess) return pn_status(e);
    return check_err(N);
}

flups_status flups_pnet_predict(flups_pnet N, const double* rho, double rho0, const double* p_n, const double* p_nm1,
                                double* p_hat) {
    NvtxRange nvtx_("flups_pnet_predict");
    flups_status st = check_fields(N, rho, rho0, p_n, p_nm1);
    if (st != FLUPS_OK) return st;
    if (!p_hat || !al16(p_hat) || p_hat == p_n || p_hat == p_nm1 || p_hat == rho) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    forward_hidden(N, rho, rho0, p_n, p_nm1);
    ConvArgs a = conv_args(N);
    a.in = N->act[2];
    a.w = N->wf + 3 * (size_t)PN_WPK;
    a.wtc = N->wtf + 3 * (size_t)PN_TCW;
    a.bias = N->w + lay_b(3);
    a.pn = p_n; a.pnm1 = p_nm1; a.phat = p_hat;
    conv<1, 1>(N, a);
    return pn_status(cudaGetLastError());
}

// Forward through the loss; with train != 0 also the backward pass and one Adam step.
static flups_status pnet_loss(flups_pnet N, const double* rho, double rho0, const double* p_n, const double* p_nm1,
                              const double* p_next, int train, float lr, double* loss) {
    flups_status st = check_fields(N, rho, rho0, p_n, p_nm1);
    if (st != FLUPS_OK) return st;
    if (!p_next || !al16(p_next)) return FLUPS_EINVAL;
    if (train && (!(lr >= 0.0f) || !std::isfinite(lr))) return FLUPS_EINVAL;
    PnGuard dg(N->dev);
    forward_hidden(N, rho, rho0, p_n, p_nm1);
    ConvArgs a = conv_args(N);
    a.in = N->act[2];
    a.w = N->wf + 3 * (size_t)PN_WPK;
    a.wtc = N->wtf + 3 * (size_t)PN_TCW;
    a.bias = N->w + lay_b(3);
    a.pn = p_n; a.pnm1 = p_nm1; a.pnext = p_next;
    a.out = N->dy;
    a.gscale = 2.0 / (double)N->n;
    conv<1, 2>(N, a);
    pk_begin(N, PK_UPDATE);
    k_pnet_fin<<<1, 1024, 0, N->stream>>>(N->red, N->last_red, N->sc, 1, 1.0 / (double)N->n);
    pk_end(N);
    N->launches++;
    if (train) {
        // dZ of layer l+1's input side: g = conv(dZ_{l+1}, W_{l+1} reversed) masked by act_l > 0
        const __nv_bfloat16* dzl = N->dy;
        for (int l = 3; l >= 1; --l) {
            __nv_bfloat16* gout = N->g[l & 1];
            ConvArgs b = conv_args(N);
            b.in = dzl;
            b.w = N->wb + (size_t)l * PN_WPK;
            b.wtc = N->wtb + (size_t)l * PN_TCW;
            b.mask = N->act[l - 1];
            b.out = gout;
            conv<2, 3>(N, b);
            wgrad(N, l, dzl, N->act[l - 1]);
            dzl = gout;
        }
        wgrad(N, 0, dzl, N->feat);
        dim3 rg((PN_PART + 255) / 256, 4);
        pk_begin(N, PK_UPDATE);
        k_pnet_reduce<<<rg, 256, 0, N->stream>>>(N->part, N->ncta, N->grad);
        pk_end(N);
        N->launches++;
        pack(N, 1, lr);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pn_status(e);
    if (loss) {
        e = cudaMemcpyAsync(N->sc_host, N->sc, 3 * sizeof(double), cudaMemcpyDeviceToHost, N->stream);
        if (e != cudaSuccess) return pn_status(e);
        st = check_err(N);
        if (st != FLUPS_OK) return st;
        *loss = N->sc_host[2];
        if (!std::isfinite(*loss)) return FLUPS_ENONFINITE;
    }
    return FLUPS_OK;
}

flups_status flups_pnet_train_step(flups_pnet N, const double* rho, double rho0, const double* p_n,
                                   const double* p_nm1, const double* p_next, float lr, double* loss) {
    NvtxRange nvtx_("flups_pnet_train_step");
    return pnet_loss(N, rho, rho0, p_n, p_nm1, p_next, 1, lr, loss);
}

flups_status flups_pnet_eval_loss(flups_pnet N, const double* rho, double rho0, const double* p_n,
                                  const double* p_nm1, const double* p_next, double* loss) {
    if (!loss) return FLUPS_EINVAL;
    return pnet_loss(N, rho, rho0, p_n, p_nm1, p_next, 0, 0.0f, loss);
}

unsigned long long flups_pnet_launch_count(flups_pnet N) { return N ? N->launches : 0; }

}  // extern "C"
