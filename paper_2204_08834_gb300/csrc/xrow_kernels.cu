// xrow_kernels.cu - kernels and launchers of the FP32 transforms along x held in registers
// (FluTAS Sec. 3.3.1, steps 2 and 8: the real-to-complex transform of each x row of the
// right-hand side, and its inverse into p), for rows of nx = 2M points with M = N1 N2 a power
// of two from 64 to 1024.  The row layout, the forward and inverse bodies and their algebra
// are in xrow.cuh (shared with the defect pass and the batched ensemble stages).
#include "blocksum.cuh"
#include "flups_impl.cuh"
#include "fp_bits.cuh"
#include "regfft.cuh"
#include "xrow.cuh"

namespace {

template <int N1, int N2, bool STATS>
__global__ void __launch_bounds__(XROW_THREADS, N1 >= 32 ? 2 : 3) k_xrow4_fwd(const double* __restrict__ f, float2* __restrict__ S,
                                                                             Geo g, const float2* __restrict__ tw,
                                                                             const float2* __restrict__ twr, int nrows,
                                                                             double* __restrict__ part) {
    xrow4_fwd_body<N1, N2, STATS>(blockIdx.x, f, S, g, tw, twr, nrows, part);
}

template <int N1, int N2, int ACC, bool MEAN, bool SUBM, bool F32>
__global__ void __launch_bounds__(XROW_THREADS) k_xrow4_inv(const float2* __restrict__ S, double* __restrict__ p,
                                                          float* __restrict__ p32, Geo g,
                                                          const float2* __restrict__ tw,
                                                          const float2* __restrict__ twr, int nrows,
                                                          DevScalars* __restrict__ sc, double* __restrict__ part) {
    xrow4_inv_body<N1, N2, ACC, MEAN, SUBM, F32>(blockIdx.x, S, p, p32, g, tw, twr, nrows, sc, part);
}

// The first inverse into the binary32 iterate (p = x with the mean's sums, stored in p32): four
// CTAs per SM where the rows are short enough (M <= 256).
template <int N1, int N2>
__global__ void __launch_bounds__(XROW_THREADS, N1 <= 16 ? 4 : 2) k_xrow4_inv_first32(
        const float2* __restrict__ S, double* __restrict__ p, float* __restrict__ p32, Geo g,
        const float2* __restrict__ tw, const float2* __restrict__ twr, int nrows, DevScalars* __restrict__ sc,
        double* __restrict__ part) {
    xrow4_inv_body<N1, N2, 0, true, false, true>(blockIdx.x, S, p, p32, g, tw, twr, nrows, sc, part);
}

template <typename K, typename... A>
bool launch_rows(K kern, size_t smem, int nrows, int B, cudaStream_t st, A... args) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    kern<<<(nrows + B - 1) / B, XROW_THREADS, smem, st>>>(args...);
    return true;
}

template <int N1, int N2>
bool fwd_n(flups_plan P, const double* f, const Geo& g, bool stats) {
    using X = XRow<N1, N2>;
    const int nrows = g.ny * g.nz;
    if (stats)
        return launch_rows(k_xrow4_fwd<N1, N2, true>, X::SMEM, nrows, X::B, P->stream, f, (float2*)P->spec, g,
                           (const float2*)P->twx, (const float2*)P->twxr, nrows, P->part);
    return launch_rows(k_xrow4_fwd<N1, N2, false>, X::SMEM, nrows, X::B, P->stream, f, (float2*)P->spec, g,
                       (const float2*)P->twx, (const float2*)P->twxr, nrows, P->part);
}

template <int N1, int N2>
bool inv_n(flups_plan P, double* p, const Geo& g, int mode) {
    using X = XRow<N1, N2>;
    const int nrows = g.ny * g.nz;
    const float2* S = (const float2*)P->spec;
    const float2* tw = (const float2*)P->twx;
    const float2* twr = (const float2*)P->twxr;
    float* p32 = P->p32;
    switch (mode) {
        case 0: return launch_rows(k_xrow4_inv<N1, N2, 0, true, false, false>, X::SMEM, nrows, X::B, P->stream, S,
                                   p, p32, g, tw, twr, nrows, P->sc, P->part);
        case 1: return launch_rows(k_xrow4_inv<N1, N2, 1, false, true, false>, X::SMEM, nrows, X::B, P->stream, S,
                                   p, p32, g, tw, twr, nrows, P->sc, P->part);
        case 2: return launch_rows(k_xrow4_inv<N1, N2, 1, false, false, false>, X::SMEM, nrows, X::B, P->stream, S,
                                   p, p32, g, tw, twr, nrows, P->sc, P->part);
        case 4: return p32 && launch_rows(k_xrow4_inv_first32<N1, N2>, X::SMEM, nrows, X::B,
                                          P->stream, S, p, p32, g, tw, twr, nrows, P->sc, P->part);
        case 5: return p32 && launch_rows(k_xrow4_inv<N1, N2, 1, false, true, true>, X::SMEM, nrows, X::B,
                                          P->stream, S, p, p32, g, tw, twr, nrows, P->sc, P->part);
        default: return launch_rows(k_xrow4_inv<N1, N2, 0, false, false, false>, X::SMEM, nrows, X::B, P->stream,
                                    S, p, p32, g, tw, twr, nrows, P->sc, P->part);
    }
}

}  // namespace

// Rows per CTA of the register row kernels for M = nx / 2, or 0 where they do not apply.
int xrow4_rows(int M) {
    switch (M) {
        case 64: return XRow<8, 8>::B;
        case 128: return XRow<16, 8>::B;
        case 256: return XRow<16, 16>::B;
        case 512: return XRow<32, 16>::B;
        case 1024: return XRow<32, 32>::B;
        default: return 0;
    }
}

bool launch_xrow4_fwd(flups_plan P, const double* f, const Geo& g, bool stats) {
    switch (g.M) {
        case 64: return fwd_n<8, 8>(P, f, g, stats);
        case 128: return fwd_n<16, 8>(P, f, g, stats);
        case 256: return fwd_n<16, 16>(P, f, g, stats);
        case 512: return fwd_n<32, 16>(P, f, g, stats);
        case 1024: return fwd_n<32, 32>(P, f, g, stats);
        default: return false;
    }
}

bool launch_xrow4_inv(flups_plan P, double* p, const Geo& g, int mode) {
    switch (g.M) {
        case 64: return inv_n<8, 8>(P, p, g, mode);
        case 128: return inv_n<16, 8>(P, p, g, mode);
        case 256: return inv_n<16, 16>(P, p, g, mode);
        case 512: return inv_n<32, 16>(P, p, g, mode);
        case 1024: return inv_n<32, 32>(P, p, g, mode);
        default: return false;
    }
}
