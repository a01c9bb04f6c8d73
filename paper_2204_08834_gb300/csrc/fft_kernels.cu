// fft_kernels.cu - transforms and z solves of the eigen-expansion Poisson solver
// (FluTAS Sec. 3.3.1: forward transforms along x and y, Gauss elimination along z per
// (kx, ky) or a third transform along z when z is periodic, inverse y and x).
//
// One batched, shared-memory Stockham engine (radix 8/4/2, register-resident butterflies)
// serves every direction.  A CTA stages a tile of B independent lines in shared memory as
// [n][c] (line index c fastest, pitch B+1), so that
//   * x lines (rows of the field, contiguous in HBM) are read coalesced along x and
//     transposed into the tile on the way in,
//   * y and z lines (columns of the spectrum) are read as B consecutive kx values
//     (128-256 contiguous bytes) per row at stride ldS or ny*ldS.
// The real transform along x uses the half-length complex FFT with the standard
// even/odd split (z_n = x_{2n} + i x_{2n+1}) and a post/pre-processing twiddle pass.
// Transforms are unnormalised; the whole 1/(M ny nz) (or 1/(M ny) with walls) factor is
// folded into the eigenvalue / tridiagonal tables, M = nx/2.
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "flups_impl.cuh"
#include "tma_pipe.cuh"
#include "fp_bits.cuh"
#include "blocksum.cuh"
#include "xrow.cuh"

namespace {

// ------------------------------------------------------------------ complex helpers
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// a * w (forward) or a * conj(w) (inverse)
template <bool INV, typename C> __device__ __forceinline__ C ctw(C a, C w) {
    C r;
    if (INV) { r.x = a.x * w.x + a.y * w.y; r.y = a.y * w.x - a.x * w.y; }
    else     { r.x = a.x * w.x - a.y * w.y; r.y = a.x * w.y + a.y * w.x; }
    return r;
}
// a * (-i) forward, a * (+i) inverse
template <bool INV, typename C> __device__ __forceinline__ C cmi(C a) {
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C* v) {
    C t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = cmi<INV>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

// 8-point DFT as two 4-point DFTs (even/odd inputs) and the W_8^k combination.
template <bool INV, typename C> __device__ __forceinline__ void dft8(C* v) {
    typedef decltype(v[0].x) T;
    const T r = (T)0.70710678118654752440;
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    C t1, t2, t3;
    if (INV) {  // W^-1 = (r, r), W^-2 = i, W^-3 = (-r, r)
        t1.x = r * (o1.x - o1.y); t1.y = r * (o1.x + o1.y);
        t2.x = -o2.y; t2.y = o2.x;
        t3.x = -r * (o3.x + o3.y); t3.y = r * (o3.x - o3.y);
    } else {    // W^1 = (r, -r), W^2 = -i, W^3 = (-r, -r)
        t1.x = r * (o1.x + o1.y); t1.y = r * (o1.y - o1.x);
        t2.x = o2.y; t2.y = -o2.x;
        t3.x = r * (o3.y - o3.x); t3.y = -r * (o3.x + o3.y);
    }
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

// 3-point DFT: y0 = a+b+c, y1,2 = a - (b+c)/2 -/+ i (sqrt3/2)(b-c) (forward; signs flip inverse).
template <bool INV, typename C> __device__ __forceinline__ void dft3(C* v) {
    typedef decltype(v[0].x) T;
    const T h = (T)0.86602540378443864676;
    const C a = v[0], b = v[1], c = v[2];
    const C sbc = cadd(b, c), dbc = csub(b, c);
    C m;
    m.x = a.x - (T)0.5 * sbc.x;
    m.y = a.y - (T)0.5 * sbc.y;
    C r;                     // forward: -i h (b - c); inverse: +i h (b - c)
    if (INV) { r.x = -h * dbc.y; r.y = h * dbc.x; } else { r.x = h * dbc.y; r.y = -h * dbc.x; }
    v[0] = cadd(a, sbc);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dftR(C* v) {
    if (R == 2) dft2<INV>(v);
    else if (R == 3) dft3<INV>(v);
    else if (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else dft8<INV>(v);
}

// One Stockham radix-R pass over B lines of length N held in shared memory as
// s[n * pitch + c].  Butterfly j (0 <= j < N/R) of line c reads n = j + r N/R and writes
// n = (j - k) R + k + r Ns with k = j mod Ns, after the twiddles W_{Ns R}^{k r}.
// The CTA has nthr = B N / E threads (N >= E): thread tid always works on line
// c = tid mod B and on butterflies j = tid / B + t N/E, t < E/R, so every index is a
// per-thread base plus a compile-time multiple of a stride.
template <typename C, int E, int R, bool INV>
__device__ __forceinline__ void stockham_pass(C* s, int pitch, int lgB, int N, int Ns,
                                              const C* __restrict__ tw) {
    constexpr int S = E / R;
    const int tid = threadIdx.x;
    const int cc = tid & ((1 << lgB) - 1), j0 = tid >> lgB;
    const int NE = N / E, NR = N / R, twstep = N / (Ns * R);
    C v[S][R];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const C* src = s + (j0 + t * NE) * pitch + cc;
#pragma unroll
        for (int r = 0; r < R; ++r) v[t][r] = src[r * NR * pitch];
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const int jj = j0 + t * NE;
        const int k = (Ns & (Ns - 1)) == 0 ? (jj & (Ns - 1)) : jj % Ns;
        if (Ns > 1) {
            // W^{k r} for r = 1..R-1 from one table entry W^k by repeated multiplication
            // (a few ulp in FP32, exact enough for the refined solve; table lookups in FP64)
            if (sizeof(v[0][0].x) == 4) {
                const C w1 = __ldg(&tw[k * twstep]);
                C wr = w1;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    v[t][r] = ctw<INV>(v[t][r], wr);
                    if (r + 1 < R) wr = ctw<false>(wr, w1);
                }
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) v[t][r] = ctw<INV>(v[t][r], __ldg(&tw[k * r * twstep]));
            }
        }
        dftR<R, INV>(v[t]);
        C* dst = s + ((jj - k) * R + k) * pitch + cc;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r * Ns * pitch] = v[t][r];
    }
    __syncthreads();
}

// Full transform of length L.n on the tile (all threads of the CTA take part).
template <typename C, int E, bool INV>
__device__ __forceinline__ void fft_tile(C* s, int pitch, int lgB, const FftLen& L, const C* __restrict__ tw) {
    int Ns = 1;
    for (int st = 0; st < L.nst; ++st) {
        const int R = (int)((L.code >> (4 * st)) & 15u);
        if constexpr (E % 8 == 0) {
            if (R == 8) { stockham_pass<C, E, 8, INV>(s, pitch, lgB, L.n, Ns, tw); Ns *= R; continue; }
        }
        if constexpr (E % 3 == 0) {
            if (R == 3) { stockham_pass<C, E, 3, INV>(s, pitch, lgB, L.n, Ns, tw); Ns *= R; continue; }
        }
        if (R == 4) stockham_pass<C, E, 4, INV>(s, pitch, lgB, L.n, Ns, tw);
        else stockham_pass<C, E, 2, INV>(s, pitch, lgB, L.n, Ns, tw);
        Ns *= R;
    }
}

// x * 2^(58 - E) as a 64-bit integer, truncated toward zero, for |x| < 2^E; sh = 1017 + E.
// Built from the binary64 layout with integer operations only: the 53-bit significand is
// placed 5 bits up and shifted right by 5 - (e - sh) >= 0 (a shift of 64 or more gives 0);
// zero and subnormal inputs give 0.  The 7-point sums of such values are exact in 64-bit
// integers (|sum| < 12 * 2^58 < 2^62).
__device__ __forceinline__ long long fixq(double x, int sh) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    unsigned long long m = ((unsigned long long)(b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000ULL) << 5;
    m = e == 0 ? 0ull : m;                  // zero and subnormals give 0 at any scale
    int r = 5 - (e - sh);
    r = r < 0 ? 0 : (r > 64 ? 64 : r);
    unsigned long long v;
    asm("shr.b64 %0, %1, %2;" : "=l"(v) : "l"(m), "r"(r));
    const long long sg = b >> 63;           // 0 or -1
    return ((long long)v ^ sg) - sg;
}

// As fixq at the scale x * 2^(1075 - sh), but for values up to 2^61 (three bits of left
// shift past fixq's range); ok = false (value unusable) at or beyond 2^61 and for infinities
// and NaNs.  Integer operations only.
__device__ __forceinline__ long long fixw(double x, int sh, bool& ok) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    unsigned long long m = ((unsigned long long)(b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000ULL) << 5;
    m = e == 0 ? 0ull : m;                  // |value| = m 2^l, m < 2^58
    const int l = e - sh - 5;
    ok = e == 0 || l <= 3;
    const unsigned r = l < 0 ? (unsigned)(l < -64 ? 64 : -l) : 0u;
    const unsigned q = l > 0 ? (unsigned)(l > 3 ? 3 : l) : 0u;
    unsigned long long v;
    asm("shr.b64 %0, %1, %2;" : "=l"(v) : "l"(m), "r"(r));
    asm("shl.b64 %0, %1, %2;" : "=l"(v) : "l"(v), "r"(q));
    const long long sg = b >> 63;
    return ((long long)v ^ sg) - sg;
}

// |D| < 2^63 to binary32 from two 32-bit halves of |D| (at most two roundings, within 2^-23
// relative), with integer-to-float conversions of 32-bit values only.
__device__ __forceinline__ float i64_to_f32(long long D) {
    const unsigned long long a = D < 0 ? (unsigned long long)(-D) : (unsigned long long)D;
    const float m = fmaf(__uint2float_rn((unsigned)(a >> 32)), 4294967296.f, __uint2float_rn((unsigned)a));
    return D < 0 ? -m : m;
}

template <typename T> __device__ __forceinline__ T from_double(double x) {
    if constexpr (sizeof(T) == 4) return d2f_bits(x);
    else return x;
}
template <typename T> __device__ __forceinline__ double to_double(T x) {
    if constexpr (sizeof(T) == 4) return f2d_bits(x);
    else return x;
}

template <typename T> __device__ __forceinline__ typename cplx<T>::t mk(T a, T b) {
    typename cplx<T>::t r; r.x = a; r.y = b; return r;
}


// The residual pass (MODE 2) uses shared-memory fixed-point rows when one thread per pair
// position covers B = E rows of one plane: E = 8, M a multiple of 32 up to 512, ny % 8 == 0.
__host__ __device__ __forceinline__ bool xres_tiled(int E, int B, int M, int ny) {
    return E == 8 && B == 8 && M % 32 == 0 && M <= 512 && ny % 8 == 0;
}
// Shared memory of that path: B + 2 rows of M fixed-point pairs (16 bytes each), and the B
// rows of the plane below.
__host__ __device__ __forceinline__ size_t xres_smem(int M) { return (size_t)18 * M * 16; }
// Planes per CTA of the z-marching defect kernel: up to 16, fewer while the grid of
// (ny / 8) x ceil(nz / kz) CTAs would hold under three waves of two CTAs on each of 152 SMs.
inline int xres_kz(int ny, int nz) {
    int kz = 16;
    while (kz > 1 && (long)(ny / 8) * ((nz + kz - 1) / kz) < 3 * 2 * 152) kz >>= 1;
    return kz;
}

__device__ __forceinline__ int ilog2_dev(int x) { return 31 - __clz(x); }

// The transform of a tile of B rows (Z in shared memory, pair index n of row c at
// s[n pitch + c]) and the real-to-complex split into the spectrum rows row0 .. row0+B-1:
// X_k = A_k + W_nx^k B_k and X_{M-k} = conj(A_k - W_nx^k B_k), k = 0..M/2, with
// A_k = (Z_k + conj Z_{M-k})/2 and B_k = (Z_k - conj Z_{M-k})/(2i).  All threads take part.
template <typename T, int E>
__device__ __forceinline__ void xfwd_tile_out(typename cplx<T>::t* s, int pitch, int lgB, const FftLen& L,
                                              const typename cplx<T>::t* __restrict__ tw,
                                              const typename cplx<T>::t* __restrict__ twr,
                                              typename cplx<T>::t* __restrict__ S, const Geo& g, int row0,
                                              int nrows) {
    typedef typename cplx<T>::t C;
    fft_tile<C, E, false>(s, pitch, lgB, L, tw);
    const int B = 1 << lgB, M = g.M, H = M / 2 + 1;
    for (int idx = threadIdx.x; idx < B * H; idx += blockDim.x) {
        const int c = idx / H, k = idx - c * H;
        const int row = row0 + c;
        if (row >= nrows) continue;
        const C zk = s[k * pitch + c];
        const C zm = s[(k == 0 ? 0 : M - k) * pitch + c];
        const T ax = (zk.x + zm.x) * (T)0.5, ay = (zk.y - zm.y) * (T)0.5;
        const T bxx = (zk.y + zm.y) * (T)0.5, byy = (zm.x - zk.x) * (T)0.5;
        const C w = __ldg(&twr[k]);
        const T tx = w.x * bxx - w.y * byy, ty = w.x * byy + w.y * bxx;
        C* out = S + (size_t)row * g.ldS;
        out[k] = mk<T>(ax + tx, ay + ty);
        if (k != M - k) out[M - k] = mk<T>(ax - tx, ty - ay);
    }
}

// ------------------------------------------------------------- forward along x (R2C)
// MODE 0: input f (FP64).  With STATS, also the partial sums
//         sum_k dzf_k sum_ij f (FP64), sum f^2 and sum f (FP32 per thread, FP64 across).
// MODE 1: input r = f - (L p + <f>_V) evaluated in FP64 on the fly (the defect of the
//         refinement), with the partial sum of r^2.
// MODE 2: the same defect on a grid with one spacing h in x, y and z: h^2 L p is an integer
//         combination of the seven p values, summed exactly in 64-bit fixed point (scale
//         2^(58-E), E from the largest exponent of p recorded when p was written), then
//         r = (f - <f>) - (2^(E-58)/h^2) S with one conversion and one FMA in FP64 (FP32 tiles
//         of 8 rows with M a multiple of 32 up to 512 and ny % 8 == 0 go to k_xres_zm instead).
// MODE 3: as MODE 2, but only the partial sums of r^2 (no transform, nothing written): the
//         stopping test of a refinement that has most likely converged.
template <typename T, int E, int MODE, bool STATS>
__device__ __forceinline__ void xfwd_body(int bx, const double* __restrict__ f, const double* __restrict__ p,
                                          typename cplx<T>::t* __restrict__ S, const Geo& g, const FftLen& L,
                                          const typename cplx<T>::t* __restrict__ tw,
                                          const typename cplx<T>::t* __restrict__ twr,
                                          const double* __restrict__ dd, int lgB, int nrows,
                                          const DevScalars* __restrict__ sc, double* __restrict__ part) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    typedef typename cplx<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    const int B = 1 << lgB, pitch = B + 1, M = g.M;
    const int row0 = bx * B, tid = threadIdx.x, nthr = blockDim.x;
    const int nx = g.nx;
    double accw = 0.0;
    float acc2 = 0.f, acc1 = 0.f;
    double mf = 0.0;
    if (MODE >= 1) mf = sc->mean_f;
    int sh = 0;
    double cfix = 0.0;
    // power-of-two spacing: r = 2^(pexp-1080)/h^2 (F - MF - S) from the exact integer difference
    // (F, MF: h^2 f and h^2 <f> at the fixed point of S), no FP64 instruction (as k_xres_zm)
    bool ipath = false;
    int shf = 0;
    long long mfq = 0;
    float rscale = 0.f;
    if (MODE >= 2) {
        const int pe_ = sc->pexp;
        sh = pe_ - 5;
        if (pe_ >= 2047) cfix = __longlong_as_double(0x7FF8000000000000LL);           // NaN: p not finite
        else if (pe_ - 57 >= 1) cfix = __hiloint2double((pe_ - 57) << 20, 0) * g.sx;   // 2^(pexp-1080) / h^2
        if (sizeof(T) == 4 && g.h2e != H2E_NONE && pe_ < 2047 && pe_ - 57 >= 1) {
            const int es = pe_ - 1080 - g.h2e;
            shf = sh - g.h2e;
            bool okm;
            mfq = fixw(mf, shf, okm);
            ipath = okm && es >= -126 && es <= 60;
            if (ipath) rscale = __int_as_float((es + 127) << 23);
        }
    }
    // Every thread handles exactly E elements (nthr = B M / E): compile-time trip counts let
    // the loads of a thread be issued before they are used.
    float fh = 0.f, fl = 0.f;   // FP32 mode, STATS: the plane's sum of f in binary32 pairs
    int kcur = -1;
    if (MODE == 0) {
        double2 fvs[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int idx = tid + q * nthr;
            const int c = idx / M, n = idx - c * M;
            const int row = row0 + c;
            fvs[q] = row < nrows ? __ldg(reinterpret_cast<const double2*>(f + (size_t)row * nx) + n)
                                 : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int idx = tid + q * nthr;
            const int c = idx / M, n = idx - c * M;
            const int row = row0 + c;
            const double2 fv = fvs[q];
            const C z = mk<T>(from_double<T>(fv.x), from_double<T>(fv.y));
            if (STATS && row < nrows) {
                const int k = row / g.ny;
                if constexpr (sizeof(T) == 4) {
                    // split f = xh + xl (bit operations), xh added by exact two-sums; flushed to
                    // FP64 with the plane's dzf only when the row moves to another plane
                    if (k != kcur) {
                        if (kcur >= 0) accw = fma(f2d_bits(fh) + f2d_bits(fl), __ldg(g.dzf + kcur), accw);
                        fh = fl = 0.f;
                        kcur = k;
                    }
                    float h0, l0, h1, l1;
                    split_d(fv.x, h0, l0);
                    split_d(fv.y, h1, l1);
                    two_sum_acc(fh, fl, h0);
                    two_sum_acc(fh, fl, h1);
                    fl += l0 + l1;
                } else {
                    accw = fma(fv.x + fv.y, __ldg(g.dzf + k), accw);
                }
                acc2 = fmaf((float)z.x, (float)z.x, fmaf((float)z.y, (float)z.y, acc2));
                acc1 += (float)z.x + (float)z.y;
            }
            s[n * pitch + c] = z;
        }
    } else {
#pragma unroll 2
    for (int q = 0; q < E; ++q) {
        const int idx = tid + q * nthr;
        const int c = idx / M, n = idx - c * M;
        const int row = row0 + c;
        C z = mk<T>((T)0, (T)0);
        if (row < nrows) {
            const double2 fv = __ldg(reinterpret_cast<const double2*>(f + (size_t)row * nx) + n);
            if (MODE == 0) {
                z = mk<T>(from_double<T>(fv.x), from_double<T>(fv.y));
                if (STATS) {
                    const int k = row / g.ny;
                    accw = fma(fv.x + fv.y, __ldg(g.dzf + k), accw);
                    acc2 = fmaf((float)z.x, (float)z.x, fmaf((float)z.y, (float)z.y, acc2));
                    acc1 += (float)z.x + (float)z.y;
                }
            } else if (MODE >= 2) {
                const int k = row / g.ny, j = row - k * g.ny;
                const int x0 = 2 * n;
                const double* pr = p + (size_t)row * nx;
                const double2 pc = __ldg(reinterpret_cast<const double2*>(pr) + n);
                const double pw = __ldg(pr + (wrapm(x0 - 1, nx)));
                const double pe = __ldg(pr + (wrapm(x0 + 2, nx)));
                const int jm = wrapm(j - 1, g.ny), jp = wrapm(j + 1, g.ny);
                int km, kp;
                if (g.walls) { km = k > 0 ? k - 1 : 0; kp = k < g.nz - 1 ? k + 1 : g.nz - 1; }
                else { km = (k - 1 + g.nz) % g.nz; kp = (k + 1) % g.nz; }
                const double2 ps = __ldg(reinterpret_cast<const double2*>(p + ((size_t)k * g.ny + jm) * nx) + n);
                const double2 pn = __ldg(reinterpret_cast<const double2*>(p + ((size_t)k * g.ny + jp) * nx) + n);
                const double2 pb = __ldg(reinterpret_cast<const double2*>(p + ((size_t)km * g.ny + j) * nx) + n);
                const double2 pt = __ldg(reinterpret_cast<const double2*>(p + ((size_t)kp * g.ny + j) * nx) + n);
                const long long q0 = fixq(pc.x, sh), q1 = fixq(pc.y, sh);
                long long s0 = fixq(pw, sh) + q1 + fixq(ps.x, sh) + fixq(pn.x, sh);
                long long s1 = q0 + fixq(pe, sh) + fixq(ps.y, sh) + fixq(pn.y, sh);
                int nd = 4;
                if (!g.walls || k > 0) { s0 += fixq(pb.x, sh); s1 += fixq(pb.y, sh); ++nd; }
                if (!g.walls || k < g.nz - 1) { s0 += fixq(pt.x, sh); s1 += fixq(pt.y, sh); ++nd; }
                s0 -= (long long)nd * q0;
                s1 -= (long long)nd * q1;
                bool ok0 = false, ok1 = false;
                long long F0 = 0, F1 = 0;
                if (ipath) {
                    F0 = fixw(fv.x, shf, ok0);
                    F1 = fixw(fv.y, shf, ok1);
                }
                if (ok0 && ok1)
                    z = mk<T>((T)(rscale * i64_to_f32(F0 - mfq - s0)), (T)(rscale * i64_to_f32(F1 - mfq - s1)));
                else
                    z = mk<T>(from_double<T>(fma(-cfix, __ll2double_rn(s0), fv.x - mf)),
                              from_double<T>(fma(-cfix, __ll2double_rn(s1), fv.y - mf)));
                acc2 = fmaf((float)z.x, (float)z.x, fmaf((float)z.y, (float)z.y, acc2));
            } else {
                const int k = row / g.ny, j = row - k * g.ny;
                const int x0 = 2 * n;
                const double* pr = p + (size_t)row * nx;
                const double2 pc = __ldg(reinterpret_cast<const double2*>(pr) + n);
                const double pw = __ldg(pr + (wrapm(x0 - 1, nx)));
                const double pe = __ldg(pr + (wrapm(x0 + 2, nx)));
                const int jm = wrapm(j - 1, g.ny), jp = wrapm(j + 1, g.ny);
                int km, kp;
                if (g.walls) { km = k > 0 ? k - 1 : 0; kp = k < g.nz - 1 ? k + 1 : g.nz - 1; }
                else { km = (k - 1 + g.nz) % g.nz; kp = (k + 1) % g.nz; }
                const double2 ps = __ldg(reinterpret_cast<const double2*>(p + ((size_t)k * g.ny + jm) * nx) + n);
                const double2 pn = __ldg(reinterpret_cast<const double2*>(p + ((size_t)k * g.ny + jp) * nx) + n);
                const double2 pb = __ldg(reinterpret_cast<const double2*>(p + ((size_t)km * g.ny + j) * nx) + n);
                const double2 pt = __ldg(reinterpret_cast<const double2*>(p + ((size_t)kp * g.ny + j) * nx) + n);
                const double azk = __ldg(g.az + k), czk = __ldg(g.cz + k), dk = __ldg(dd + k);
                double a0 = fma(g.sx, pw + pc.y, mf);
                a0 = fma(g.sy, ps.x + pn.x, a0);
                a0 = fma(azk, pb.x, a0);
                a0 = fma(czk, pt.x, a0);
                a0 = fma(-dk, pc.x, a0);
                double a1 = fma(g.sx, pc.x + pe, mf);
                a1 = fma(g.sy, ps.y + pn.y, a1);
                a1 = fma(azk, pb.y, a1);
                a1 = fma(czk, pt.y, a1);
                a1 = fma(-dk, pc.y, a1);
                z = mk<T>(from_double<T>(fv.x - a0), from_double<T>(fv.y - a1));
                acc2 = fmaf((float)z.x, (float)z.x, fmaf((float)z.y, (float)z.y, acc2));
            }
        }
        s[n * pitch + c] = z;
    }
    }
    if (STATS) {
        if (sizeof(T) == 4 && kcur >= 0) accw = fma(f2d_bits(fh) + f2d_bits(fl), __ldg(g.dzf + kcur), accw);
        block_sum_abc<true, true, true>(accw, acc2, acc1, part, bx);
    }
    else if (MODE >= 1) block_sum_abc<false, true, false>(0.0, acc2, 0.f, part, bx);
    if (MODE == 3) return;               // the defect norm only (the stopping test)
    __syncthreads();
    xfwd_tile_out<T, E>(s, pitch, lgB, L, tw, twr, S, g, row0, nrows);
}
template <typename T, int E, int MODE, bool STATS>
__global__ void __launch_bounds__(512) k_xfwd(const double* __restrict__ f, const double* __restrict__ p,
                                               typename cplx<T>::t* __restrict__ S, Geo g, FftLen L,
                                               const typename cplx<T>::t* __restrict__ tw,
                                               const typename cplx<T>::t* __restrict__ twr,
                                               const double* __restrict__ dd, int lgB, int nrows,
                                               const DevScalars* __restrict__ sc, double* __restrict__ part) {
    xfwd_body<T, E, MODE, STATS>(blockIdx.x, f, p, S, g, L, tw, twr, dd, lgB, nrows, sc, part);
}

// fixq of a binary32 value at sh = pexp - 5, i.e. x * 2^(1080 - pexp) truncated toward zero, with
// two binary32 products by ka = 2^a, kb = 2^b (a + b = 1080 - pexp, each within the binary32
// exponent range) and one conversion to a 64-bit integer.  Both products are exact while the
// value stays a normal number; a product in the subnormal range has magnitude below 2^-126 and
// truncates to 0 either way, and |x| < 2^(pexp - 1022) keeps the result below 2^58.
__device__ __forceinline__ long long fixf(float x, float ka, float kb) {
    return __float2ll_rz(__fmul_rn(__fmul_rn(x, ka), kb));
}

// The FP32 refinement's exact defect on one-spacing grids (MODE 2: with the forward transform
// of r; MODE 3: the partial sums of r^2 only), marching up through z.  A CTA owns a block of
// E = 8 consecutive rows j0 .. j0+7 of the planes k0 .. k1-1, one thread per pair position n.
// The 7-point sum S of p is exact in 64-bit fixed point (fixq at the scale of the largest
// exponent of p).  On a grid whose spacing is a power of two, h^2 (f - <f>) is taken to the
// same fixed point (F, MF: truncated, 2^-58 of the scale of p or finer), so
// r = 2^(pexp-1080)/h^2 (F - MF - S) needs no FP64 instruction: the integer difference is
// exact and is rounded to binary32 once, and the power-of-two scale is exact.  Points whose F
// would reach 2^61, and every point when h^2 <f> would, take r = (f - <f>) - cfix S in FP64.
// Each p is converted to fixed point about once: plane k+1's centre rows are converted, serve
// as the upper z neighbours of plane k, then move into shared memory (with the two y-halo
// rows, converted there) as the centre of plane k+1, while the centre of plane k stays in
// registers as the lower neighbour of plane k+1: 1.25 conversions per point plus one plane
// per chunk of kz planes (3.25 when every row converts its own z neighbours).  With MODE 2 the
// transform tile reuses the shared rows after each plane's stencil.  part[b]
// (b = blockIdx.x + gridDim.x blockIdx.y) takes the block sums of r^2.
// PT = float: p is the first FP32 iterate held in binary32 (rows of nx values, as p), read at
// 4 bytes a point and taken to fixed point by fixf, the same integers as fixq of its binary64
// value.
// fq (one-spacing power-of-two grids, may be null): MODE 2 writes F - MF of every point it owns
// (fqs[0] = the scale pexp it used, fqs[1] set where some point had no integer form); MODE 3
// reads it instead of f, skipping f's conversion, when fqs shows the same scale and no gap.
// As a body: G groups of M threads (the CTA's G row blocks j0 = (bx G + grp) 8 .. +7, consecutive,
// of the planes by kz .. by kz + kz - 1), each group with its own shared rows; the Stockham tail
// transforms the 8 G rows together (the four-step tail, N1 > 0, takes G = 1).  part[pidx]
// takes the CTA's sum of r^2.
template <int E, int MODE, int N1, int N2, typename PT>
__device__ __forceinline__ void xres_zm_body(int bx, int by, int G, const double* __restrict__ f,
                                             const PT* __restrict__ p, float2* __restrict__ S, const Geo& g,
                                             const FftLen& L, const float2* __restrict__ tw,
                                             const float2* __restrict__ twr, int kz,
                                             const DevScalars* __restrict__ sc, double* __restrict__ part,
                                             int pidx, long long* __restrict__ fq, int* __restrict__ fqs) {
    static_assert(E == 8, "one pair position per thread over 8 rows");
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = g.M, grp = threadIdx.x / M, n = threadIdx.x - grp * M, pitch = E * G + 1;
    longlong2* Q = reinterpret_cast<longlong2*>(smraw) + (size_t)grp * (E + 2) * M;
    float2* s = reinterpret_cast<float2*>(smraw);
    const int j0 = (bx * G + grp) * E, k0 = by * kz, jc = bx * G * E;
    const int k1 = min(k0 + kz, g.nz);
    const double mf = sc->mean_f;
    const int pe_ = sc->pexp, sh = pe_ - 5;
    double cfix = 0.0;
    if (pe_ >= 2047) cfix = __longlong_as_double(0x7FF8000000000000LL);           // NaN: p not finite
    else if (pe_ - 57 >= 1) cfix = __hiloint2double((pe_ - 57) << 20, 0) * g.sx;   // 2^(pexp-1080) / h^2
    bool ipath = false;
    int shf = 0;
    long long mfq = 0;
    float rscale = 0.f;
    if (g.h2e != H2E_NONE && pe_ < 2047 && pe_ - 57 >= 1) {
        const int es = pe_ - 1080 - g.h2e;
        shf = sh - g.h2e;
        bool okm;
        mfq = fixw(mf, shf, okm);
        ipath = okm && es >= -126 && es <= 60;
        if (ipath) rscale = __int_as_float((es + 127) << 23);
    }
    constexpr bool PF = sizeof(PT) == 4;
    typedef typename cplx<PT>::t P2T;        // one pair of p: float2 or double2
    float ka = 1.f, kb = 1.f;                // fixf's factors (PF): 2^a 2^b = 2^(1080 - pexp)
    if (PF) {
        const int s2 = 1080 - pe_, a2 = s2 >> 1;
        ka = __int_as_float((min(max(a2, -126), 127) + 127) << 23);
        kb = __int_as_float((min(max(s2 - a2, -126), 127) + 127) << 23);
    }
    auto fix2 = [&](const P2T& v) {
        if constexpr (PF) return make_longlong2(fixf(v.x, ka, kb), fixf(v.y, ka, kb));
        else return make_longlong2(fixq(v.x, sh), fixq(v.y, sh));
    };
    const P2T* P2 = reinterpret_cast<const P2T*>(p);
    const bool fq_write = MODE == 2 && PF && fq != nullptr;   // the first defect only
    const bool fq_read = MODE == 3 && fq != nullptr && ipath && fqs[1] == 0 && fqs[0] == pe_;
    if (fq_write && pidx == 0 && threadIdx.x == 0) fqs[0] = ipath ? pe_ : -1;
    bool fq_gap = false;
    // the raw 64-bit values of f (binary64) or of F - MF (fq_read), [row][M] pairs either way
    const longlong2* FR = fq_read ? reinterpret_cast<const longlong2*>(fq) : reinterpret_cast<const longlong2*>(f);
    const int nw_ = n == 0 ? M - 1 : n - 1, ne_ = n + 1 == M ? 0 : n + 1;
    auto prow = [&](int k, int j) { return P2 + ((size_t)k * g.ny + j) * M + n; };
    // LO[c M + n]: the centre of the plane below (thread n alone reads and writes column n)
    longlong2* LO = reinterpret_cast<longlong2*>(smraw) + (size_t)G * (E + 2) * M + (size_t)grp * E * M;
    // the centre of plane k0 with its y halo into shared memory, the plane below into LO
#pragma unroll
    for (int r = 0; r < E + 2; ++r) {
        Q[r * M + n] = fix2(__ldg(prow(k0, wrapm(j0 - 1 + r, g.ny))));
    }
    {
        const bool has = !g.walls || k0 > 0;
        const int kb = k0 == 0 ? g.nz - 1 : k0 - 1;
#pragma unroll
        for (int c = 0; c < E; ++c) {
            longlong2 q = make_longlong2(0, 0);
            if (has) q = fix2(__ldg(prow(kb, j0 + c)));
            LO[c * M + n] = q;
        }
    }
    float acc2 = 0.f;
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const bool hb = !g.walls || k > 0, ht = !g.walls || k < g.nz - 1;
        const int kt = k + 1 == g.nz ? 0 : k + 1;
        const long long nd = 4 + (hb ? 1 : 0) + (ht ? 1 : 0);
        const size_t row0 = (size_t)k * g.ny + j0;
        // every global load of the plane first (p of plane k+1 with its y halo, f of plane k),
        // so that one memory latency per plane is exposed
        P2T pu[E + 2];
        longlong2 fr[E];
#pragma unroll
        for (int c = 0; c < E; ++c) fr[c] = __ldg(FR + (row0 + c) * M + n);
        const bool more = k + 1 < k1;
#pragma unroll
        for (int r = 0; r < E + 2; ++r) {
            pu[r] = P2T{};
            if ((r >= 1 && r <= E && ht) || more) pu[r] = __ldg(prow(kt, wrapm(j0 - 1 + r, g.ny)));
        }
        float2 zr[E];
        longlong2 uq[E];                      // plane k+1's centre rows, converted once
#pragma unroll
        for (int c = 0; c < E; ++c) {
            const longlong2 qc = Q[(c + 1) * M + n], qs = Q[c * M + n], qn = Q[(c + 2) * M + n];
            const long long qw = Q[(c + 1) * M + nw_].y, qe = Q[(c + 1) * M + ne_].x;
            const longlong2 ql = LO[c * M + n];
            uq[c] = fix2(pu[c + 1]);           // 0 for a wall's ghost
            long long s0 = qw + qc.y + qs.x + qn.x - nd * qc.x + ql.x + uq[c].x;
            long long s1 = qc.x + qe + qs.y + qn.y - nd * qc.y + ql.y + uq[c].y;
            LO[c * M + n] = qc;                // the lower neighbour of plane k+1
            bool ok0 = false, ok1 = false;
            long long F0 = 0, F1 = 0;            // F - MF
            if (fq_read) {
                ok0 = ok1 = true;
                F0 = fr[c].x;
                F1 = fr[c].y;
            } else if (ipath) {
                F0 = fixw(__longlong_as_double(fr[c].x), shf, ok0) - mfq;
                F1 = fixw(__longlong_as_double(fr[c].y), shf, ok1) - mfq;
            }
            if (ok0 && ok1) {
                zr[c] = make_float2(rscale * i64_to_f32(F0 - s0), rscale * i64_to_f32(F1 - s1));
            } else {
                zr[c] = make_float2(d2f_bits(fma(-cfix, __ll2double_rn(s0), __longlong_as_double(fr[c].x) - mf)),
                                    d2f_bits(fma(-cfix, __ll2double_rn(s1), __longlong_as_double(fr[c].y) - mf)));
            }
            if (fq_write) {
                fq_gap |= !(ok0 && ok1);
                reinterpret_cast<longlong2*>(fq)[(row0 + c) * M + n] = make_longlong2(F0, F1);
            }
            acc2 = fmaf(zr[c].x, zr[c].x, fmaf(zr[c].y, zr[c].y, acc2));
        }
        __syncthreads();                      // every read of plane k's shared rows is done
        if (MODE == 2 && N1 == 0) {
#pragma unroll
            for (int c = 0; c < E; ++c) s[n * pitch + grp * E + c] = zr[c];
            __syncthreads();
            xfwd_tile_out<float, E>(s, pitch, ilog2_dev(E * G), L, tw, twr, S, g, (int)((size_t)k * g.ny + jc),
                                    g.ny * g.nz);
            __syncthreads();                  // the tile is read out: the rows of plane k+1 may go in
        } else if constexpr (MODE == 2 && N1 > 0) {
            // the register four-step rows, in their own area T after the rows of Q and LO: the
            // 8 rows go through T (pitch TP, 8 (mod 16) when N2 = 8 so that the two rows of a
            // half-warp fall on distinct banks) to the 8 N2 threads that hold z[N2 n1 + t] of
            // row c = tid / N2 (the other warps pass the barriers only); plane k+1 moves into
            // Q first, so that its prefetched rows are not held through the transform
            constexpr int TP = N1 * N2 + (N2 == 8 ? 8 : 0);
            float2* T = reinterpret_cast<float2*>(smraw + (size_t)G * xres_smem(M));
#pragma unroll
            for (int c = 0; c < E; ++c) T[c * TP + n] = zr[c];
            if (more) {
#pragma unroll
                for (int r = 0; r < E + 2; ++r)
                    Q[r * M + n] = r >= 1 && r <= E ? uq[r - 1] : fix2(pu[r]);
            }
            __syncthreads();
            const bool active = n < E * N2;
            const int c = n / N2, t = n % N2;
            float2 v[N1];
            if (active) {
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) v[n1] = T[c * TP + N2 * n1 + t];
            }
            __syncthreads();                  // T is read out: the exchange may take its place
            xrow4_fwd_tail<N1, N2>(v, T, active ? c : 0, t, active, true, tw, twr,
                                   S + (row0 + (active ? c : 0)) * g.ldS);
            continue;                         // T is next written after the next plane's stencil
        }
        if (more) {
#pragma unroll
            for (int r = 0; r < E + 2; ++r)
                Q[r * M + n] = r >= 1 && r <= E ? uq[r - 1] : fix2(pu[r]);
            __syncthreads();
        }
    }
    if (fq_write && __any_sync(0xffffffffu, fq_gap) && (threadIdx.x & 31) == 0) atomicExch(fqs + 1, 1);
    block_sum_abc<false, true, false>(0.0, acc2, 0.f, part, pidx);
}

template <int E, int MODE, int N1, int N2, typename PT>
__global__ void __launch_bounds__(512, 1) k_xres_zm(const double* __restrict__ f, const PT* __restrict__ p,
                                                   float2* __restrict__ S, Geo g, FftLen L,
                                                   const float2* __restrict__ tw, const float2* __restrict__ twr,
                                                   int kz, const DevScalars* __restrict__ sc,
                                                   double* __restrict__ part, long long* __restrict__ fq,
                                                   int* __restrict__ fqs) {
    xres_zm_body<E, MODE, N1, N2, PT>(blockIdx.x, blockIdx.y, 1, f, p, S, g, L, tw, twr, kz, sc, part,
                                      blockIdx.y * gridDim.x + blockIdx.x, fq, fqs);
}

// ------------------------------------------------------------- inverse along x (C2R)
// ACC = 0: p = x (FP64 store);  ACC = 1: p += x (FP64 defect-correction update).
// MEAN (with ACC = 0): also the partial sums of dzf * p for the volume-weighted mean of the
// first FP32 iterate, whose rounding leaves a constant of order eps32 |p| that the
// residual cannot see; SUBM (with ACC = 1) removes that constant in the first update.
template <typename T, int E, int ACC, bool MEAN, bool SUBM>
__device__ __forceinline__ void xinv_body(int bx, const typename cplx<T>::t* __restrict__ S, double* __restrict__ p,
                                          const Geo& g, const FftLen& L, const typename cplx<T>::t* __restrict__ tw,
                                          const typename cplx<T>::t* __restrict__ twr, int lgB, int nrows,
                                          DevScalars* __restrict__ sc, double* __restrict__ part) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    typedef typename cplx<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    const int B = 1 << lgB, pitch = B + 1, M = g.M;
    const int row0 = bx * B, tid = threadIdx.x, nthr = blockDim.x;
    const int H = M / 2 + 1;
    // Z_k = A_k + i B_k, Z_{M-k} = conj(A_k) + i conj(B_k) with A_k = (X_k + conj X_{M-k})/2,
    // B_k = (X_k - conj X_{M-k}) conj(W_nx^k)/2; X_0 and X_M are taken real.
    // B H = nthr (E/2) + B elements: at most E/2 + 1 per thread, loaded before use.
    constexpr int QH = E / 2 + 1;
    C xks[QH], xms[QH];
#pragma unroll
    for (int q = 0; q < QH; ++q) {
        const int idx = tid + q * nthr;
        const int c = idx / H, k = idx - c * H;
        const int row = row0 + c;
        xks[q] = mk<T>((T)0, (T)0);
        xms[q] = xks[q];
        if (idx < B * H && row < nrows) {
            const C* in = S + (size_t)row * g.ldS;
            xks[q] = in[k];
            xms[q] = in[M - k];
        }
    }
#pragma unroll
    for (int q = 0; q < QH; ++q) {
        const int idx = tid + q * nthr;
        if (idx >= B * H) break;
        const int c = idx / H, k = idx - c * H;
        C xk = xks[q], xm = xms[q];
        if (k == 0) { xk.y = (T)0; xm.y = (T)0; }
        const T ax = (xk.x + xm.x) * (T)0.5, ay = (xk.y - xm.y) * (T)0.5;
        const T dx = (xk.x - xm.x) * (T)0.5, dy = (xk.y + xm.y) * (T)0.5;
        const C w = __ldg(&twr[k]);
        const T bxx = dx * w.x + dy * w.y, byy = dy * w.x - dx * w.y;
        s[k * pitch + c] = mk<T>(ax - byy, ay + bxx);
        if (k != 0 && k != M - k) s[(M - k) * pitch + c] = mk<T>(ax + byy, bxx - ay);
    }
    __syncthreads();
    fft_tile<C, E, true>(s, pitch, lgB, L, tw);
    const int nx = g.nx;
    double accw = 0.0;
    float mh = 0.f, ml = 0.f;   // FP32 mode: the plane's sum of p in binary32 pairs (two-sums)
    int kcur = -1;
    int emax = 0;       // largest binary64 exponent field written (FP32 mode: scale of the next defect)
    T msub = (T)0;
    if (SUBM) msub = (T)sc->mean_p;
    double2 pold[ACC ? E : 1];
    if (ACC) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int idx = tid + q * nthr;
            const int c = idx / M, n = idx - c * M;
            const int row = row0 + c;
            pold[q] = row < nrows ? *(reinterpret_cast<const double2*>(p + (size_t)row * nx) + n)
                                  : make_double2(0.0, 0.0);
        }
    }
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int idx = tid + q * nthr;
        const int c = idx / M, n = idx - c * M;
        const int row = row0 + c;
        if (row >= nrows) continue;
        C z = s[n * pitch + c];
        if (SUBM) { z.x -= msub; z.y -= msub; }
        double2* dst = reinterpret_cast<double2*>(p + (size_t)row * nx) + n;
        double2 o;
        if (ACC) {
            o = pold[ACC ? q : 0];
            o.x += to_double<T>(z.x);
            o.y += to_double<T>(z.y);
        } else {
            o.x = to_double<T>(z.x);
            o.y = to_double<T>(z.y);
            if (MEAN) {
                if constexpr (sizeof(T) == 4) {
                    // flushed to FP64 with the plane's dzf only when the row moves to another plane
                    const int k = row / g.ny;
                    if (k != kcur) {
                        if (kcur >= 0) accw = fma(f2d_bits(mh) + f2d_bits(ml), __ldg(g.dzf + kcur), accw);
                        mh = ml = 0.f;
                        kcur = k;
                    }
                    two_sum_acc(mh, ml, (float)z.x);
                    two_sum_acc(mh, ml, (float)z.y);
                } else {
                    accw = fma(o.x + o.y, __ldg(g.dzf + row / g.ny), accw);
                }
            }
        }
        *dst = o;
        if (sizeof(T) == 4) {
            const int ex = (int)((__double_as_longlong(o.x) >> 52) & 0x7FF);
            const int ey = (int)((__double_as_longlong(o.y) >> 52) & 0x7FF);
            emax = max(emax, max(ex, ey));
        }
    }
    if (sizeof(T) == 4) {
        emax = __reduce_max_sync(0xffffffffu, emax);
        if ((tid & 31) == 0) atomicMax(&sc->pexp, emax);
    }
    if (MEAN) {
        if (sizeof(T) == 4 && kcur >= 0) accw = fma(f2d_bits(mh) + f2d_bits(ml), __ldg(g.dzf + kcur), accw);
        block_sum_abc<true, false, false>(accw, 0.f, 0.f, part, bx);
    }
}
template <typename T, int E, int ACC, bool MEAN, bool SUBM>
__global__ void __launch_bounds__(512) k_xinv(const typename cplx<T>::t* __restrict__ S, double* __restrict__ p,
                                               Geo g, FftLen L, const typename cplx<T>::t* __restrict__ tw,
                                               const typename cplx<T>::t* __restrict__ twr, int lgB, int nrows,
                                               DevScalars* __restrict__ sc, double* __restrict__ part) {
    xinv_body<T, E, ACC, MEAN, SUBM>(blockIdx.x, S, p, g, L, tw, twr, lgB, nrows, sc, part);
}

// -------------------------------------------- x transforms with Neumann or Dirichlet ends
// KIND 1 (Neumann at both ends): X_k = sum_j x_j cos(pi k (2j+1)/(2 nx)), k < nx (DCT-II);
// KIND 2 (Dirichlet at both ends): Y_k = sum_j x_j sin(pi (k+1)(2j+1)/(2 nx)), the DCT-II of
// (-1)^j x_j read backwards (DST-II).  Makhoul's construction: v_n = x_{2n}, v_{nx-1-n} = x_{2n+1};
// V = the real FFT of v (half-length complex FFT and split, as in k_xfwd); X_k = Re(q_k V_k) and
// X_{nx-k} = -Im(q_k V_k) with q_k = exp(-i pi k/(2 nx)), k = 0..M.  The nx real coefficients go
// to S[row][k] as (X_k, 0).  INV: V_k = conj(q_k) (X_k - i X_{nx-k}) (X_nx = 0), the merge and
// half-length inverse FFT of k_xinv, and the inverse permutation; unnormalised like k_xinv (a
// round trip gives M x).  ACC = 1 adds the result to p.
// KIND 3 (Neumann at the low face, Dirichlet at the high face): X_k = sum_j x_j
// cos(pi (2j+1)(2k+1)/(4 nx)) (DCT-IV); KIND 4 (Dirichlet low, Neumann high): the sine kind
// (DST-IV) = (-1)^k DCT-IV of x read backwards.  An nx/2-point complex FFT of
// u_m = (x_{2m} + i x_{nx-1-2m}) exp(-i pi (4m+1)/(4 nx)), then y_k = U_k exp(-i pi k/nx),
// X_{2k} = Re y_k, X_{nx-1-2k} = -Im y_k.  The kind is its own inverse up to nx/2 = M, the
// scaling of the other x transforms, so INV runs the same steps on the coefficients.
template <typename T, int E, int KIND, int ACC>
__device__ __forceinline__ void xdct4_row_tile(typename cplx<T>::t* __restrict__ S, const double* __restrict__ fin,
                                               double* __restrict__ pout, bool inv, const Geo& g, const FftLen& L,
                                               const typename cplx<T>::t* __restrict__ tw,
                                               const typename cplx<T>::t* __restrict__ pre,
                                               const typename cplx<T>::t* __restrict__ post, int lgB, int nrows,
                                               unsigned char* smraw) {
    typedef typename cplx<T>::t C;
    C* s = reinterpret_cast<C*>(smraw);
    T* sT = reinterpret_cast<T*>(smraw);
    const int B = 1 << lgB, pitch = B + 1, M = g.M, nx = g.nx;
    const int row0 = blockIdx.x * B, tid = threadIdx.x, nthr = blockDim.x;
    constexpr bool SINE = KIND == 4;
    for (int idx = tid; idx < B * M; idx += nthr) {
        const int c = idx / M, n = idx - c * M;
        const int row = row0 + c;
        double a = 0.0, b = 0.0;                          // x_{2n}, x_{2n+1}
        if (row < nrows) {
            if (!inv) {
                const double2 xv = __ldg(reinterpret_cast<const double2*>(fin + (size_t)row * nx) + n);
                a = xv.x;
                b = xv.y;
            } else {
                const C* in = S + (size_t)row * g.ldS;
                if (g.xpack) {   // X_k is the k-th real of the row
                    a = (double)reinterpret_cast<const T*>(in)[2 * n];
                    b = (double)reinterpret_cast<const T*>(in)[2 * n + 1];
                } else {
                    a = (double)in[2 * n].x;
                    b = (double)in[2 * n + 1].x;
                }
            }
        }
        // x_{2n} is u_n's real part (cosine kind) and x_{2n+1} = x_{nx-1-2m} for m = M-1-n its
        // imaginary part; the sine kind reads x backwards, which swaps the two.
        sT[(n * pitch + c) * 2 + (SINE ? 1 : 0)] = from_double<T>(a);
        sT[((M - 1 - n) * pitch + c) * 2 + (SINE ? 0 : 1)] = from_double<T>(b);
    }
    __syncthreads();
    for (int idx = tid; idx < B * M; idx += nthr) {
        const int c = idx % B, m = idx / B;
        const C w = __ldg(&pre[m]);
        const C u = s[m * pitch + c];
        s[m * pitch + c] = mk<T>(u.x * w.x - u.y * w.y, u.x * w.y + u.y * w.x);
    }
    __syncthreads();
    fft_tile<C, E, false>(s, pitch, lgB, L, tw);
    for (int idx = tid; idx < B * M; idx += nthr) {
        const int c = idx / M, k = idx - c * M;
        const int row = row0 + c;
        if (row >= nrows) continue;
        const C w = __ldg(&post[k]);
        const C U = s[k * pitch + c];
        const T yr = U.x * w.x - U.y * w.y, yi = U.x * w.y + U.y * w.x;
        const T xe = yr, xo = SINE ? yi : -yi;           // X_{2k}, X_{nx-1-2k} (sine: times (-1)^index)
        if (!inv) {
            C* out = S + (size_t)row * g.ldS;
            if (g.xpack) {
                reinterpret_cast<T*>(out)[2 * k] = xe;
                reinterpret_cast<T*>(out)[nx - 1 - 2 * k] = xo;
            } else {
                out[2 * k] = mk<T>(xe, (T)0);
                out[nx - 1 - 2 * k] = mk<T>(xo, (T)0);
            }
        } else {
            double* dst = pout + (size_t)row * nx;
            double ve = to_double<T>(xe), vo = to_double<T>(xo);
            if (ACC) { ve += dst[2 * k]; vo += dst[nx - 1 - 2 * k]; }
            dst[2 * k] = ve;
            dst[nx - 1 - 2 * k] = vo;
        }
    }
}

template <typename T, int E, int KIND, bool INV, int ACC>
__global__ void __launch_bounds__(512) k_xdct(typename cplx<T>::t* __restrict__ S, const double* __restrict__ fin,
                                               double* __restrict__ pout, Geo g, FftLen L,
                                               const typename cplx<T>::t* __restrict__ tw,
                                               const typename cplx<T>::t* __restrict__ twr,
                                               const typename cplx<T>::t* __restrict__ twq, int lgB, int nrows) {
    typedef typename cplx<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    if constexpr (KIND >= 3) {   // twr: pre-twiddles, twq: post-twiddles of the DCT-IV kind
        xdct4_row_tile<T, E, KIND, ACC>(S, fin, pout, INV, g, L, tw, twr, twq, lgB, nrows, smraw);
    } else {
        C* s = reinterpret_cast<C*>(smraw);
        T* sT = reinterpret_cast<T*>(smraw);
        const int B = 1 << lgB, pitch = B + 1, M = g.M, nx = g.nx;
        const int row0 = blockIdx.x * B, tid = threadIdx.x, nthr = blockDim.x;
        const int H = M / 2 + 1;
        // v_m lives in packed element m/2 of line c, real part for even m
        auto vat = [&](int m, int c) -> T& { return sT[((m >> 1) * pitch + c) * 2 + (m & 1)]; };
        if constexpr (!INV) {
            for (int idx = tid; idx < B * M; idx += nthr) {
                const int c = idx / M, n = idx - c * M;
                const int row = row0 + c;
                const double2 xv = row < nrows ? __ldg(reinterpret_cast<const double2*>(fin + (size_t)row * nx) + n)
                                               : make_double2(0.0, 0.0);
                vat(n, c) = from_double<T>(xv.x);
                vat(nx - 1 - n, c) = from_double<T>(KIND == 2 ? -xv.y : xv.y);
            }
            __syncthreads();
            fft_tile<C, E, false>(s, pitch, lgB, L, tw);
            for (int idx = tid; idx < B * H; idx += nthr) {
                const int c = idx / H, k = idx - c * H;
                const int row = row0 + c;
                if (row >= nrows) continue;
                const C zk = s[k * pitch + c];
                const C zm = s[(k == 0 ? 0 : M - k) * pitch + c];
                const T ax = (zk.x + zm.x) * (T)0.5, ay = (zk.y - zm.y) * (T)0.5;
                const T bxx = (zk.y + zm.y) * (T)0.5, byy = (zm.x - zk.x) * (T)0.5;
                const C w = __ldg(&twr[k]);
                const T tx = w.x * bxx - w.y * byy, ty = w.x * byy + w.y * bxx;
                C* out = S + (size_t)row * g.ldS;
                auto put = [&](int idx, T v) {           // X_idx: (X, 0), or the idx-th real when packed
                    if (g.xpack) reinterpret_cast<T*>(out)[idx] = v;
                    else out[idx] = mk<T>(v, (T)0);
                };
                auto emit = [&](int kk, T vx, T vy) {   // X_kk and X_{nx-kk} from V_kk
                    const C q = __ldg(&twq[kk]);
                    const T re = q.x * vx - q.y * vy, im = q.x * vy + q.y * vx;
                    put(KIND == 2 ? nx - 1 - kk : kk, re);
                    if (kk != 0 && kk != M) put(KIND == 2 ? kk - 1 : nx - kk, -im);
                };
                emit(k, ax + tx, ay + ty);                         // V_k
                if (k != M - k) emit(M - k, ax - tx, ty - ay);     // V_{M-k} (k = 0: V_M)
            }
        } else {
            for (int idx = tid; idx < B * H; idx += nthr) {
                const int c = idx / H, k = idx - c * H;
                const int row = row0 + c;
                C xk = mk<T>((T)0, (T)0), xm = xk;
                if (row < nrows) {
                    const C* in = S + (size_t)row * g.ldS;
                    auto X = [&](int j) -> T {
                        const int jj = KIND == 2 ? nx - 1 - j : j;
                        return g.xpack ? reinterpret_cast<const T*>(in)[jj] : in[jj].x;
                    };
                    auto vk = [&](int kk) -> C {                       // conj(q_kk) (X_kk - i X_{nx-kk})
                        const T a = X(kk), b = kk == 0 ? (T)0 : X(nx - kk);
                        const C q = __ldg(&twq[kk]);
                        return mk<T>(q.x * a - q.y * b, -(q.x * b + q.y * a));
                    };
                    xk = vk(k);
                    xm = vk(M - k);
                }
                if (k == 0) { xk.y = (T)0; xm.y = (T)0; }
                const T ax = (xk.x + xm.x) * (T)0.5, ay = (xk.y - xm.y) * (T)0.5;
                const T dx = (xk.x - xm.x) * (T)0.5, dy = (xk.y + xm.y) * (T)0.5;
                const C w = __ldg(&twr[k]);
                const T bxx = dx * w.x + dy * w.y, byy = dy * w.x - dx * w.y;
                s[k * pitch + c] = mk<T>(ax - byy, ay + bxx);
                if (k != 0 && k != M - k) s[(M - k) * pitch + c] = mk<T>(ax + byy, bxx - ay);
            }
            __syncthreads();
            fft_tile<C, E, true>(s, pitch, lgB, L, tw);
            for (int idx = tid; idx < B * M; idx += nthr) {
                const int c = idx / M, n = idx - c * M;
                const int row = row0 + c;
                if (row >= nrows) continue;
                const T a = vat(n, c), b = vat(nx - 1 - n, c);
                double2* dst = reinterpret_cast<double2*>(pout + (size_t)row * nx) + n;
                double2 o = make_double2(to_double<T>(a), to_double<T>(KIND == 2 ? -b : b));
                if (ACC) { const double2 old = *dst; o.x += old.x; o.y += old.y; }
                *dst = o;
            }
        }
    }
}

// ------------------------------------------- y transforms with Neumann or Dirichlet ends
// On complex columns (kx fixed): the cosine (KIND 1) or sine (KIND 2) series of the real and of
// the imaginary part together, from one complex FFT of length ny of the permuted column
// (v_m = z_{2m}, v_{ny-1-m} = z_{2m+1}; odd entries negated for KIND 2):
//   X_k = (Re(q_k (V_k + conj V_{ny-k})) + i Im(q_k (V_k - conj V_{ny-k}))) / 2,  q_k = exp(-i pi k/(2 ny)),
// stored backwards for KIND 2.  INV: V_k = conj(q_k)[(Re X_k - i Re X_{ny-k}) + i (Im X_k - i Im X_{ny-k})],
// the unnormalised inverse FFT and the inverse permutation.  A tile is B columns of one plane.
template <typename T, int E, int KIND, bool INV>
__global__ void __launch_bounds__(1024) k_ydct(typename cplx<T>::t* __restrict__ S, Geo g, FftLen L,
                                               const typename cplx<T>::t* __restrict__ tw,
                                               const typename cplx<T>::t* __restrict__ twq, int lgB, int ncols) {
    typedef typename cplx<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    const int B = 1 << lgB, pitch = B + 1;
    const int kxa = blockIdx.x * B;
    C* base = S + (size_t)blockIdx.y * g.ny * g.ldS + kxa;
    const int N = g.ny, tid = threadIdx.x, nthr = blockDim.x;
    const int c = tid & (B - 1), j0 = tid >> lgB, NE = N / E;
    const bool live = kxa + c < ncols;
    auto vpos = [&](int j) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); };   // z_j -> v_vpos(j)
    const int HP = N / 2 + 1;
    {
        C r[E];
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int j = j0 + t * NE;
            const int src = INV && KIND == 2 ? N - 1 - j : j;
            r[t] = live ? base[(size_t)src * g.ldS + c] : mk<T>((T)0, (T)0);
        }
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int j = j0 + t * NE;
            C z = r[t];
            if (!INV && KIND == 2 && (j & 1)) { z.x = -z.x; z.y = -z.y; }
            s[(INV ? j : vpos(j)) * pitch + c] = z;
        }
    }
    __syncthreads();
    if (!INV) fft_tile<C, E, false>(s, pitch, lgB, L, tw);
    __syncthreads();
    for (int idx = tid; idx < B * HP; idx += nthr) {   // the pair (k, N-k) of one column
        const int cc = idx % B, k = idx / B;
        const int km = k == 0 ? 0 : N - k;
        const C a = s[k * pitch + cc], b = s[km * pitch + cc];
        const C qk = __ldg(&twq[k]);
        if (!INV) {
            // X_k from (V_k, V_{N-k}); X_{N-k} from (V_{N-k}, V_k)
            const T sx = a.x + b.x, sy = a.y - b.y, dx = a.x - b.x, dy = a.y + b.y;
            const C xk = mk<T>((T)0.5 * (qk.x * sx - qk.y * sy), (T)0.5 * (qk.x * dy + qk.y * dx));
            if (k != 0 && k != km) {
                const C qm = __ldg(&twq[km]);
                const T sx2 = b.x + a.x, sy2 = b.y - a.y, dx2 = b.x - a.x, dy2 = b.y + a.y;
                s[km * pitch + cc] = mk<T>((T)0.5 * (qm.x * sx2 - qm.y * sy2), (T)0.5 * (qm.x * dy2 + qm.y * dx2));
            }
            s[k * pitch + cc] = xk;
        } else {
            // V_k = conj(q_k) (Re X_k - i Re X_{N-k}) + i conj(q_k) (Im X_k - i Im X_{N-k}), X_N = 0
            const C bb = k == 0 ? mk<T>((T)0, (T)0) : b;
            auto vk = [&](C q, C x1, C x2) -> C {
                const C A = mk<T>(q.x * x1.x - q.y * x2.x, -(q.x * x2.x + q.y * x1.x));   // conj(q)(x1.x - i x2.x)
                const C Bq = mk<T>(q.x * x1.y - q.y * x2.y, -(q.x * x2.y + q.y * x1.y));  // conj(q)(x1.y - i x2.y)
                return mk<T>(A.x - Bq.y, A.y + Bq.x);                                     // A + i B
            };
            const C vkk = vk(qk, a, bb);
            if (k != 0 && k != km) s[km * pitch + cc] = vk(__ldg(&twq[km]), bb, a);
            s[k * pitch + cc] = vkk;
        }
    }
    __syncthreads();
    if (INV) {
        fft_tile<C, E, true>(s, pitch, lgB, L, tw);
        __syncthreads();
    }
    if (live) {
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int j = j0 + t * NE;
            if (!INV) {
                base[(size_t)(KIND == 2 ? N - 1 - j : j) * g.ldS + c] = s[j * pitch + c];
            } else {
                C z = s[vpos(j) * pitch + c];
                if (KIND == 2 && (j & 1)) { z.x = -z.x; z.y = -z.y; }
                base[(size_t)j * g.ldS + c] = z;
            }
        }
    }
}

// ------------------------------------- y transforms with mixed ends (Neumann / Dirichlet)
// KIND 3 (Neumann low, Dirichlet high: DCT-IV) and KIND 4 (Dirichlet low, Neumann high: DST-IV)
// on complex columns: the real and the imaginary part of a column are two real sequences of
// length ny, each transformed with the ny/2-point construction of xdct4_row_tile; a tile of B
// complex columns is 2B sub-columns of ny/2 complex points (2c: real parts, 2c+1: imaginary
// parts).  The kind is its own inverse up to ny/2; INV doubles the result so that a round trip
// gives ny z like the other y transforms.
template <typename T, int E, int KIND, bool INV>
__global__ void __launch_bounds__(1024) k_ydct4(typename cplx<T>::t* __restrict__ S, Geo g, FftLen L2,
                                                const typename cplx<T>::t* __restrict__ tw2,
                                                const typename cplx<T>::t* __restrict__ pre,
                                                const typename cplx<T>::t* __restrict__ post, int lgB, int ncols) {
    typedef typename cplx<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    T* sT = reinterpret_cast<T*>(smraw);
    constexpr bool SINE = KIND == 4;
    const int B = 1 << lgB, B2 = 2 * B, pitch = B2 + 1;
    const int N = g.ny, H = N / 2, tid = threadIdx.x, nthr = blockDim.x;
    const int kxa = blockIdx.x * B;
    C* base = S + (size_t)blockIdx.y * g.ny * g.ldS + kxa;
    for (int idx = tid; idx < B * N; idx += nthr) {
        const int c = idx % B, j = idx / B;
        const C z = kxa + c < ncols ? base[(size_t)j * g.ldS + c] : mk<T>((T)0, (T)0);
        // element j of a sequence: even j = 2m -> u_m real part (sine: imaginary), odd j -> u_m
        // with m = (N-1-j)/2, imaginary part (sine: real)
        const bool even = (j & 1) == 0;
        const int m = even ? (j >> 1) : ((N - 1 - j) >> 1);
        const int comp = (even != SINE) ? 0 : 1;
        sT[(m * pitch + 2 * c) * 2 + comp] = z.x;
        sT[(m * pitch + 2 * c + 1) * 2 + comp] = z.y;
    }
    __syncthreads();
    for (int idx = tid; idx < B2 * H; idx += nthr) {
        const int cc = idx % B2, m = idx / B2;
        const C w = __ldg(&pre[m]);
        const C u = s[m * pitch + cc];
        s[m * pitch + cc] = mk<T>(u.x * w.x - u.y * w.y, u.x * w.y + u.y * w.x);
    }
    __syncthreads();
    fft_tile<C, E, false>(s, pitch, lgB + 1, L2, tw2);
    __syncthreads();
    const T sc = INV ? (T)2 : (T)1;
    for (int idx = tid; idx < B * H; idx += nthr) {
        const int c = idx % B, k = idx / B;
        if (kxa + c >= ncols) continue;
        const C w = __ldg(&post[k]);
        const C Ua = s[k * pitch + 2 * c], Ub = s[k * pitch + 2 * c + 1];
        const T ar = Ua.x * w.x - Ua.y * w.y, ai = Ua.x * w.y + Ua.y * w.x;
        const T br = Ub.x * w.x - Ub.y * w.y, bi = Ub.x * w.y + Ub.y * w.x;
        base[(size_t)(2 * k) * g.ldS + c] = mk<T>(sc * ar, sc * br);
        base[(size_t)(N - 1 - 2 * k) * g.ldS + c] = SINE ? mk<T>(sc * ai, sc * bi) : mk<T>(-sc * ai, -sc * bi);
    }
}

// ------------------------------------------------------- column transform along y
// TAIL = false: a tile of B consecutive kx columns of plane blockIdx.y.
// TAIL = true : the Nyquist column kx = M of B consecutive planes (blockIdx.x * B + c), so
//               that this ragged column is transformed by full tiles too.
template <typename T, int E, bool INV, bool TAIL>
__device__ __forceinline__ void ycol_body(int bx, int by, typename cplx<T>::t* __restrict__ S, const Geo& g,
                                          const FftLen& L, const typename cplx<T>::t* __restrict__ tw, int lgB,
                                          int kx0) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    typedef typename cplx<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    const int B = 1 << lgB, pitch = B + 1;
    const size_t plane = (size_t)g.ny * g.ldS;
    C* base;
    size_t cs;
    int ncol;
    if (TAIL) {
        base = S + (size_t)bx * B * plane + g.M;
        cs = plane;
        ncol = min(B, g.nz - (int)bx * B);
    } else {
        const int kxa = kx0 + bx * B;
        base = S + (size_t)by * plane + kxa;
        cs = 1;
        ncol = min(B, g.M - kxa);   // kx = M is the TAIL launch's
    }
    const int tid = threadIdx.x, N = g.ny;
    // thread tid owns line c = tid mod B and rows j0 + t N/E, t < E (nthr * E == B * N)
    const int c = tid & (B - 1), j0 = tid >> lgB, NE = N / E;
    const bool live = c < ncol;
    {   // every thread issues its E loads before touching shared memory
        C r[E];
        const C* src = base + (size_t)j0 * g.ldS + c * cs;
#pragma unroll
        for (int t = 0; t < E; ++t) r[t] = live ? src[(size_t)t * NE * g.ldS] : mk<T>((T)0, (T)0);
#pragma unroll
        for (int t = 0; t < E; ++t) s[(j0 + t * NE) * pitch + c] = r[t];
    }
    __syncthreads();
    fft_tile<C, E, INV>(s, pitch, lgB, L, tw);
    if (live) {
        C* dst = base + (size_t)j0 * g.ldS + c * cs;
#pragma unroll
        for (int t = 0; t < E; ++t) dst[(size_t)t * NE * g.ldS] = s[(j0 + t * NE) * pitch + c];
    }
}
template <typename T, int E, bool INV, bool TAIL>
__global__ void __launch_bounds__(1024) k_ycol(typename cplx<T>::t* __restrict__ S, Geo g, FftLen L,
                                               const typename cplx<T>::t* __restrict__ tw, int lgB, int kx0) {
    ycol_body<T, E, INV, TAIL>(blockIdx.x, blockIdx.y, S, g, L, tw, lgB, kx0);
}

// -------------------------------------- periodic z: forward z FFT, divide, inverse z FFT
// lam tables hold eigenvalue / norm; the (0,0,0) mode is set to zero (zero-mean p).
// TAIL = false: B consecutive kx columns at ky = blockIdx.y; TAIL = true: the Nyquist column
// kx = M at B consecutive ky (blockIdx.x * B + c).
template <typename T, int E, bool TAIL>
__device__ __forceinline__ void zper_body(int bx, int by, typename cplx<T>::t* __restrict__ S, const Geo& g,
                                          const FftLen& L, const typename cplx<T>::t* __restrict__ tw,
                                          const T* __restrict__ lamx, const T* __restrict__ lamy,
                                          const T* __restrict__ lamz, int lgB, int kx0) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    typedef typename cplx<T>::t C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = reinterpret_cast<C*>(smraw);
    const int B = 1 << lgB, pitch = B + 1;
    const size_t zs = (size_t)g.ny * g.ldS;
    C* base;
    size_t cs;
    int ncol, kxa, ky0;
    if (TAIL) {
        ky0 = bx * B;
        kxa = g.M;
        base = S + (size_t)ky0 * g.ldS + g.M;
        cs = g.ldS;
        ncol = min(B, g.ny - ky0);
    } else {
        ky0 = by;
        kxa = kx0 + bx * B;
        base = S + (size_t)ky0 * g.ldS + kxa;
        cs = 1;
        ncol = min(B, g.M - kxa);   // kx = M is the TAIL launch's
    }
    const int tid = threadIdx.x, N = g.nz;
    const int c = tid & (B - 1), j0 = tid >> lgB, NE = N / E;
    const bool live = c < ncol;
    {
        C r[E];
        const C* src = base + (size_t)j0 * zs + c * cs;
#pragma unroll
        for (int t = 0; t < E; ++t) r[t] = live ? src[(size_t)t * NE * zs] : mk<T>((T)0, (T)0);
#pragma unroll
        for (int t = 0; t < E; ++t) s[(j0 + t * NE) * pitch + c] = r[t];
    }
    __syncthreads();
    fft_tile<C, E, false>(s, pitch, lgB, L, tw);
    {
        const int cc = min(c, ncol - 1);
        const T lxy = TAIL ? __ldg(&lamx[kxa]) + __ldg(&lamy[ky0 + cc]) : __ldg(&lamx[kxa + cc]) + __ldg(&lamy[ky0]);
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int k = j0 + t * NE;
            const T lam = lxy + __ldg(&lamz[k]);
            const T inv = lam != (T)0 ? (T)1 / lam : (T)0;
            C v = s[k * pitch + c];
            v.x *= inv;
            v.y *= inv;
            s[k * pitch + c] = v;
        }
    }
    __syncthreads();
    fft_tile<C, E, true>(s, pitch, lgB, L, tw);
    if (live) {
        C* dst = base + (size_t)j0 * zs + c * cs;
#pragma unroll
        for (int t = 0; t < E; ++t) dst[(size_t)t * NE * zs] = s[(j0 + t * NE) * pitch + c];
    }
}
template <typename T, int E, bool TAIL>
__global__ void __launch_bounds__(1024) k_zper(typename cplx<T>::t* __restrict__ S, Geo g, FftLen L,
                                               const typename cplx<T>::t* __restrict__ tw,
                                               const T* __restrict__ lamx, const T* __restrict__ lamy,
                                               const T* __restrict__ lamz, int lgB, int kx0) {
    zper_body<T, E, TAIL>(blockIdx.x, blockIdx.y, S, g, L, tw, lamx, lamy, lamz, lgB, kx0);
}

// ------------------------------------- persistent, double-buffered column transforms
// FP32 column passes (y transform, or periodic z: transform, divide, inverse transform)
// with a persistent grid: each CTA owns a sequence of tiles (B consecutive kx columns by N
// rows) and keeps two tile buffers in shared memory.  While the threads transform tile i in
// place, the next tile streams into the other buffer by cp.async.bulk row copies (B
// complex = 128 bytes per row, 16-byte aligned) that complete on an mbarrier.  Tile rows are
// stored with coalesced 128-byte writes.  Every mbarrier wait is bounded: on time-out the
// CTA records an error and leaves (after a bounded wait for its own copies in flight).
// The TMA and mbarrier helpers are in tma_pipe.cuh.

// Self-test of the bounded wait (mbar_wait_bounded): one thread waits on an mbarrier that nothing ever
// arrives at, gives up after `limit` polls, records err = 3 and returns (no trap, no hang).
__global__ void k_selftest_wait(int limit, int* __restrict__ err) {
    __shared__ __align__(8) unsigned long long m;
    if (threadIdx.x == 0) mbar_init(&m, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait_bounded(&m, 0, limit)) atomicExch(err, 3);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&m)) : "memory");
    }
}

// KIND 0: y transform (INV picks the direction); KIND 1: periodic z solve.
template <int KIND, bool INV>
__global__ void __launch_bounds__(1024, 1) k_cols_pipe(float2* __restrict__ S, const __grid_constant__ CUtensorMap tm,
                                                       Geo g, FftLen L, const float2* __restrict__ tw,
                                                       const float* __restrict__ lamx, const float* __restrict__ lamy,
                                                       const float* __restrict__ lamz, int lgB, int box_rows,
                                                       int* __restrict__ err) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    constexpr int E = 8;
    typedef float2 C;
    extern __shared__ __align__(128) unsigned char smpipe[];   // [tile 0][tile 1][2 mbarriers]
    const int B = 1 << lgB;
    const int N = KIND == 0 ? g.ny : g.nz;
    const size_t rs = KIND == 0 ? (size_t)g.ldS : (size_t)g.ny * g.ldS;    // row stride (elements)
    const int tiles_x = g.M >> lgB;
    const int ntiles = tiles_x * (KIND == 0 ? g.nz : g.ny);
    const unsigned tile_bytes = (unsigned)(N * B * sizeof(C));
    C* buf0 = reinterpret_cast<C*>(smpipe);
    C* buf1 = reinterpret_cast<C*>(smpipe + tile_bytes);
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smpipe + 2 * (size_t)tile_bytes);
    const int tid = threadIdx.x;
    const int c = tid & (B - 1), j0 = tid >> lgB, NE = N / E;

    auto tile_base = [&](int t) -> C* {
        const int tx = t % tiles_x, ty = t / tiles_x;
        return KIND == 0 ? S + (size_t)ty * g.ny * g.ldS + (size_t)tx * B : S + (size_t)ty * g.ldS + (size_t)tx * B;
    };
    auto issue = [&](int t, int b) {      // one thread: expect the tile's bytes, then TMA its boxes
        if (tid == 0) {
            C* dst = b ? buf1 : buf0;
            const int tx = t % tiles_x, ty = t / tiles_x;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&mbar[b], tile_bytes);
            for (int r0 = 0; r0 < N; r0 += box_rows) {
                if (KIND == 0) tma_load_3d(dst + r0 * B, &tm, tx * B, r0, ty, &mbar[b]);
                else tma_load_3d(dst + r0 * B, &tm, tx * B, ty, r0, &mbar[b]);
            }
        }
    };

    if (smem_u32(smpipe) & 127u) {   // TMA box destinations must be 128-byte aligned
        if (tid == 0) atomicExch(err, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    unsigned parity[2] = {0u, 0u};
    int t = blockIdx.x;
    if (t < ntiles) issue(t, 0);
    bool pending_other = false;
    for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
        const int b = it & 1;
        const int tn = t + gridDim.x;
        if (tn < ntiles) issue(tn, b ^ 1);
        pending_other = tn < ntiles;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&mbar[b], parity[b]));
        parity[b] ^= 1u;
        if (!ok) {   // leave only after (bounded) waits for both buffers' copies
            if (tid == 0) atomicExch(err, 1);
            mbar_wait_bounded(&mbar[b], parity[b] ^ 1u);
            if (pending_other) mbar_wait_bounded(&mbar[b ^ 1], parity[b ^ 1]);
            return;
        }
        C* s = b ? buf1 : buf0;
        if (KIND == 0) {
            fft_tile<C, E, INV>(s, B, lgB, L, tw);
        } else {
            fft_tile<C, E, false>(s, B, lgB, L, tw);
            const int tx = t % tiles_x, ky = t / tiles_x;
            const float lxy = __ldg(&lamx[tx * B + c]) + __ldg(&lamy[ky]);
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const int k = j0 + q * NE;
                const float lam = lxy + __ldg(&lamz[k]);
                const float inv = lam != 0.f ? 1.f / lam : 0.f;
                C v = s[k * B + c];
                v.x *= inv;
                v.y *= inv;
                s[k * B + c] = v;
            }
            __syncthreads();
            fft_tile<C, E, true>(s, B, lgB, L, tw);
        }
        C* dst = tile_base(t) + (size_t)j0 * rs + c;
#pragma unroll
        for (int q = 0; q < E; ++q) dst[(size_t)q * NE * rs] = s[(j0 + q * NE) * B + c];
        __syncthreads();
    }
}

// ------------------------------------------ z walls: Gauss elimination (Thomas) along z
// One thread per (kx, ky) column; neighbouring threads take neighbouring kx, so every row
// access of a warp is a contiguous run.  tri = [a_k, b_k, c_k] / norm.  The forward
// multipliers c'_k go to a scratch array, the eliminated right-hand side d'_k overwrites
// the spectrum in place, then the back substitution overwrites it with the solution.
// Column (0, 0) is singular: its row 0 is dropped, P_0 = 0, and the column is shifted
// to zero dzf-weighted mean.
template <typename T>
__device__ __forceinline__ void ztri_body(int bx, typename cplx<T>::t* __restrict__ S, T* __restrict__ cps,
                                          const Geo& g, const T* __restrict__ lamx, const T* __restrict__ lamy,
                                          const T* __restrict__ tri) {
    if (g.skip && *g.skip) return;   // graph-capturable solve: this member already converged
    typedef typename cplx<T>::t C;
    const int ncols = g.nxh * g.ny;
    const int col = bx * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const int ky = col / g.nxh, kx = col - ky * g.nxh;
    const int nz = g.nz;
    const T* ta = tri;
    const T* tb = tri + nz;
    const T* tc = tri + 2 * nz;
    const size_t zs = (size_t)g.ny * g.ldS;
    C* x = S + (size_t)ky * g.ldS + kx;
    T* cp = cps + col;
    const size_t cs = (size_t)ncols;
    const bool sing = (col == 0) && g.sing00;   // (kx, ky) = (0, 0) has lam_x + lam_y = 0
    const T lam = sing ? (T)0 : __ldg(&lamx[kx]) + __ldg(&lamy[ky]);
    const int k0 = sing ? 1 : 0;
    // Singular column: remove the dzf-weighted mean of F over z first (= nx ny <f>_V in the
    // unnormalised spectrum), so that dropping row 0 solves L p = f - <f>_V for any f (R3).
    C fmean = mk<T>((T)0, (T)0);
    if (sing) {
        double sw = 0.0, sx0 = 0.0, sy0 = 0.0;
        for (int k = 0; k < nz; ++k) {
            const C F = x[k * zs];
            const double w = g.dzf[k];
            sw += w;
            sx0 += w * (double)F.x;
            sy0 += w * (double)F.y;
        }
        fmean = mk<T>((T)(sx0 / sw), (T)(sy0 / sw));
    }
    // Both sweeps take the column in chunks of ZQ rows whose loads are issued before the
    // chunk's recurrence steps (the steps depend on each other, the loads do not).
    constexpr int ZQ = 8;
    T cprev = (T)0;
    C dprev = mk<T>((T)0, (T)0);
    for (int kb = k0; kb < nz; kb += ZQ) {
        C Fq[ZQ];
#pragma unroll
        for (int q = 0; q < ZQ; ++q) Fq[q] = kb + q < nz ? x[(size_t)(kb + q) * zs] : mk<T>((T)0, (T)0);
#pragma unroll
        for (int q = 0; q < ZQ; ++q) {
            const int k = kb + q;
            if (k >= nz) break;
            const T a = k > k0 ? __ldg(&ta[k]) : (T)0;
            const T m = (__ldg(&tb[k]) + lam) - a * cprev;
            const T inv = (T)1 / m;
            C F = Fq[q];
            F.x -= fmean.x;
            F.y -= fmean.y;
            cprev = __ldg(&tc[k]) * inv;
            dprev = mk<T>((F.x - a * dprev.x) * inv, (F.y - a * dprev.y) * inv);
            cp[(size_t)k * cs] = cprev;
            x[(size_t)k * zs] = dprev;
        }
    }
    C xv = dprev;
    T sx = (T)0, sy = (T)0;
    if (sing) { const T w = (T)g.dzf[nz - 1]; sx = w * xv.x; sy = w * xv.y; }
    for (int kt = nz - 2; kt >= k0; kt -= ZQ) {
        T cq[ZQ];
        C dq[ZQ];
#pragma unroll
        for (int q = 0; q < ZQ; ++q) {
            const int k = kt - q;
            cq[q] = k >= k0 ? cp[(size_t)k * cs] : (T)0;
            dq[q] = k >= k0 ? x[(size_t)k * zs] : mk<T>((T)0, (T)0);
        }
#pragma unroll
        for (int q = 0; q < ZQ; ++q) {
            const int k = kt - q;
            if (k < k0) break;
            xv = mk<T>(dq[q].x - cq[q] * xv.x, dq[q].y - cq[q] * xv.y);
            x[(size_t)k * zs] = xv;
            if (sing) { const T w = (T)g.dzf[k]; sx += w * xv.x; sy += w * xv.y; }
        }
    }
    if (sing) {
        x[0] = mk<T>((T)0, (T)0);
        T sw = (T)0;
        for (int k = 0; k < nz; ++k) sw += (T)g.dzf[k];
        const T mx = sx / sw, my = sy / sw;
        for (int k = 0; k < nz; ++k) {
            C v = x[k * zs];
            v.x -= mx;
            v.y -= my;
            x[k * zs] = v;
        }
    }
}
template <typename T>
__global__ void __launch_bounds__(128) k_ztri(typename cplx<T>::t* __restrict__ S, T* __restrict__ cps, Geo g,
                                              const T* __restrict__ lamx, const T* __restrict__ lamy,
                                              const T* __restrict__ tri) {
    ztri_body<T>(blockIdx.x, S, cps, g, lamx, lamy, tri);
}

// Thomas along z for the packed all-real spectrum (Geo::xpack): complex column (m, ky) holds the
// real x modes 2m (real part) and 2m+1 (imaginary part), two real systems with the eigenvalues
// lam_x[2m] + lam_y[ky] and lam_x[2m+1] + lam_y[ky]; the real part of column 0 is the singular
// (0, 0) mode when no end is Dirichlet (mean of F removed, row 0 dropped, P_0 = 0, zero-mean shift).
template <typename T>
__global__ void __launch_bounds__(128) k_ztri_packed(typename cplx<T>::t* __restrict__ S, T* __restrict__ cps,
                                                     Geo g, const T* __restrict__ lamx, const T* __restrict__ lamy,
                                                     const T* __restrict__ tri) {
    typedef typename cplx<T>::t C;
    const int ncols = g.nxh * g.ny;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const int ky = col / g.nxh, m = col - ky * g.nxh;
    const int nz = g.nz;
    const T* ta = tri;
    const T* tb = tri + nz;
    const T* tc = tri + 2 * nz;
    const size_t zs = (size_t)g.ny * g.ldS;
    C* x = S + (size_t)ky * g.ldS + m;
    T* cp = cps + 2 * (size_t)col;
    const size_t cs = 2 * (size_t)ncols;
    const bool sing = (col == 0) && g.sing00;
    const T la = __ldg(&lamx[2 * m]) + __ldg(&lamy[ky]), lb = __ldg(&lamx[2 * m + 1]) + __ldg(&lamy[ky]);
    const int k0a = sing ? 1 : 0;
    T fmean = (T)0;
    if (sing) {
        double sw = 0.0, sx0 = 0.0;
        for (int k = 0; k < nz; ++k) {
            const double w = g.dzf[k];
            sw += w;
            sx0 += w * (double)x[k * zs].x;
        }
        fmean = (T)(sx0 / sw);
    }
    T ca = (T)0, cb = (T)0, da = (T)0, db = (T)0;
    for (int k = 0; k < nz; ++k) {
        const C F = x[k * zs];
        const T tbk = __ldg(&tb[k]), tck = __ldg(&tc[k]);
        {
            const T a_ = k > 0 ? __ldg(&ta[k]) : (T)0;
            const T inv = (T)1 / ((tbk + lb) - a_ * cb);
            cb = tck * inv;
            db = (F.y - a_ * db) * inv;
        }
        if (k >= k0a) {
            const T a_ = k > k0a ? __ldg(&ta[k]) : (T)0;
            const T inv = (T)1 / ((tbk + la) - a_ * ca);
            ca = tck * inv;
            da = ((F.x - fmean) - a_ * da) * inv;
        }
        cp[k * cs] = ca;
        cp[k * cs + 1] = cb;
        x[k * zs] = mk<T>(da, db);
    }
    T xa = da, xb = db, sxa = (T)0;
    if (sing) sxa = (T)g.dzf[nz - 1] * xa;
    for (int k = nz - 2; k >= 0; --k) {
        const C d = x[k * zs];
        xb = d.y - cp[k * cs + 1] * xb;
        if (k >= k0a) {
            xa = d.x - cp[k * cs] * xa;
            if (sing) sxa += (T)g.dzf[k] * xa;
        }
        x[k * zs] = mk<T>(k >= k0a ? xa : (T)0, xb);
    }
    if (sing) {
        T sw = (T)0;
        for (int k = 0; k < nz; ++k) sw += (T)g.dzf[k];
        const T mx = sxa / sw;
        for (int k = 0; k < nz; ++k) {
            C v = x[k * zs];
            v.x -= mx;
            x[k * zs] = v;
        }
    }
}

// Deterministic final reduction of the per-block partial sums in one launch: block g of G sums
// a contiguous chunk of the partials into fin[3 g + q]; the last block to finish (atomic
// ticket) adds the G chunk sums in a fixed order and derives the scalars.  The ticket is reset
// by that block, so the kernel can be replayed (graphs).
constexpr int FIN_THREADS = 256;
__device__ __forceinline__ void fin_block_sum(double& a, double& b, double& c, double (*red)[FIN_THREADS / 32]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = a; red[1][wid] = b; red[2][wid] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = red[0][0]; b = red[1][0]; c = red[2][0];
        for (int w = 1; w < FIN_THREADS / 32; ++w) { a += red[0][w]; b += red[1][w]; c += red[2][w]; }
    }
}

__global__ void __launch_bounds__(FIN_THREADS) k_finalize(const double* __restrict__ part, int nblk, DevScalars* sc,
                                                        int what, double nrm_w, double npts, int fixed, double thr2,
                                                        double* __restrict__ fin) {
    if (fixed && sc->done) return;   // fixed-iteration solve: the member converged earlier
    __shared__ double red[3][FIN_THREADS / 32];
    __shared__ int last;
    const int G = gridDim.x;
    const int chunk = (nblk + G - 1) / G;
    const int i0 = blockIdx.x * chunk, i1 = min(nblk, i0 + chunk);
    double a = 0.0, b = 0.0, c = 0.0;
#pragma unroll 4
    for (int i = i0 + threadIdx.x; i < i1; i += FIN_THREADS) {
        a += __ldcg(part + 3 * i + 0);
        b += __ldcg(part + 3 * i + 1);
        c += __ldcg(part + 3 * i + 2);
    }
    fin_block_sum(a, b, c, red);
    if (threadIdx.x == 0) {
        fin[3 * blockIdx.x + 0] = a;
        fin[3 * blockIdx.x + 1] = b;
        fin[3 * blockIdx.x + 2] = c;
        __threadfence();
        last = atomicAdd(&sc->fin_count, 1u) == (unsigned)(G - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    a = b = c = 0.0;
    if (threadIdx.x < G) {
        a = __ldcg(fin + 3 * threadIdx.x + 0);
        b = __ldcg(fin + 3 * threadIdx.x + 1);
        c = __ldcg(fin + 3 * threadIdx.x + 2);
    }
    __syncthreads();
    fin_block_sum(a, b, c, red);
    if (threadIdx.x == 0) {
        sc->fin_count = 0u;
        if (what == 0) {          // a = sum dzf f, b = sum f^2, c = sum f
            const double m = a * nrm_w;
            sc->mean_f = m;
            sc->f2 = b - 2.0 * m * c + npts * m * m;
        } else if (what == 1) {   // b = sum r^2
            sc->r2 = b;
            if (fixed && b <= thr2 * sc->f2) sc->done = 1;
        } else {                  // a = sum dzf p
            sc->mean_p = a * nrm_w;
        }
    }
}

// Blocks of the final reduction for nblk partials (at most FIN_THREADS).
int fin_grid(int nblk) {
    int g = nblk / 64;
    return g < 1 ? 1 : (g > FIN_THREADS ? FIN_THREADS : g);
}

// ------------------------------------------------------------------- host helpers
int ilog2i(int x) { int l = 0; while ((1 << l) < x) ++l; return l; }

// Largest CTA of the non-pipelined transform kernels: 256 threads by default (measured best
// on GB300 for the x passes at 512^3); the FLUPS_CTA_THREADS environment variable (256, 512
// or 1024) overrides it.
int cta_threads() {
    static int v = 0;
    if (!v) {
        const char* e = getenv("FLUPS_CTA_THREADS");
        const int q = e ? atoi(e) : 256;
        v = (q == 512 || q == 1024) ? q : 256;
    }
    return v;
}

// Tile width B (lines per CTA): as wide as possible up to bmax while the CTA has at most
// cta_threads() threads and 74 KB of tile (three CTAs per SM by shared memory).
int pick_lgB(int N, int csize, int E, int bmax, int ncols, int cap) {
    int B = bmax;
    const long tmax = cap > 0 ? cap : cta_threads();
    while (B > 1 && ((long)B * N / E > tmax || (long)N * (B + 1) * csize > 74 * 1024)) B >>= 1;
    while (B > 1 && B > ncols) B >>= 1;
    while ((long)B * N < E) B <<= 1;
    return ilog2i(B);
}

// Thread cap of the x passes: at most 512 threads, so that their per-thread prefetch
// registers (E complex values) fit without spills (launch bound 512: up to 128 registers).
int x_cap(int cta) { return std::min(cta > 0 ? cta : cta_threads(), 512); }

template <typename K> void allow_smem(K kern, size_t bytes = 96 * 1024) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(bytes, 96 * 1024));
}

// Elements per thread: 16 (FP32) or 8 (FP64) complex values; 4 for transforms shorter than that.
// (The radix sequences use radix 8 only for lengths >= 8, so E >= the largest radix.)
template <typename T> int e_for(int N) { return N % 3 == 0 ? 12 : (N >= 8 ? 8 : 4); }
template <typename T> struct Ebig { static const int E = 8; };

FftLen packed(FftLen L) {
    L.code = 0ull;
    for (int st = 0; st < L.nst; ++st) L.code |= (unsigned long long)L.rad[st] << (4 * st);
    return L;
}

// Tile of the pipelined kernel: B columns with B * N * 8 bytes <= 32 KB, B <= 16, B <= M (tiles
// small enough for two CTAs per SM, which overlap one's FFT with the other's copies).
int pipe_lgB(int N, int M, int kind) {
    const int l4 = cols4_lgB(N, M, kind);      // the four-step kernel's tile where it applies
    if (l4 >= 0) return l4;
    int B = 16;
    while (B > 1 && ((long)B * N * 8 > 32 * 1024 || B > M)) B >>= 1;
    return ilog2i(B);
}
// The pipelined path needs its tensor map (built with the plan), rows of at least 16 bytes
// (B >= 2) and at most 1024 threads (B N / 8).
bool pipe_ok(flups_plan P, int N, int kind) {
    if (!P->tma_ok || (N & (N - 1)) != 0) return false;
    if (cols4_lgB(N, P->M, kind) >= 0) return true;
    const int B = 1 << pipe_lgB(N, P->M, kind);
    return B >= 2 && P->M % B == 0 && (long)B * N / 8 <= 1024 && N >= 8;
}

template <int KIND, bool INV>
void run_cols_pipe(flups_plan P, float2* S, const Geo& g, const FftLen& L, const float2* tw) {
    if (launch_cols4(P, S, g, KIND, INV)) return;     // four-step kernel (cols_kernels.cu)
    const int N = KIND == 0 ? g.ny : g.nz;
    const int lgB = pipe_lgB(N, g.M, KIND), B = 1 << lgB;
    const size_t sm = 2 * (size_t)N * B * sizeof(float2) + 2 * sizeof(unsigned long long);
    auto kern = k_cols_pipe<KIND, INV>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (g.M / B) * (KIND == 0 ? g.nz : g.ny);
    // persistent CTAs: as many per SM as threads (1024 at 64 registers) and shared memory allow
    const int thr = B * N / 8;
    int per_sm = 1024 / thr;
    while (per_sm > 1 && (size_t)per_sm * (sm + 1024) > 220 * 1024) --per_sm;
    if (per_sm < 1) per_sm = 1;
    const int grid = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;
    kern<<<grid, B * N / 8, sm, P->stream>>>(S, KIND == 0 ? P->tm_y : P->tm_z, g, L, tw, (const float*)P->lamx,
                                             (const float*)P->lamy, (const float*)P->lamz, lgB, N < 256 ? N : 256,
                                             &P->sc->err);
}

template <typename T, int E, bool INV>
void run_ycol_e(flups_plan P, typename cplx<T>::t* S, const Geo& g, bool tail_col = true) {
    typedef typename cplx<T>::t C;
    const int N = g.ny;
    const int lgB = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, g.M, g.cta);
    const int B = 1 << lgB;
    const FftLen L = packed(P->ly);
    auto kern = k_ycol<T, E, INV, false>;
    auto tail = k_ycol<T, E, INV, true>;
    allow_smem(kern);
    allow_smem(tail);
    flups_prof_begin(P, sizeof(T) == 4 ? FK_YCOL32 : FK_YCOL64);
    const size_t sm = (size_t)N * (B + 1) * sizeof(C);
    if (sizeof(T) == 4 && E == 8 && pipe_ok(P, N, 0)) run_cols_pipe<0, INV>(P, (float2*)S, g, L, (const float2*)P->twy);
    else kern<<<dim3((g.M + B - 1) / B, g.nz), B * N / E, sm, P->stream>>>(S, g, L, (const C*)P->twy, lgB, 0);
    // the Nyquist column kx = M of every plane, B planes per tile
    if (tail_col) {
        const int lgT = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, g.nz, g.cta);
        const int BT = 1 << lgT;
        tail<<<dim3((g.nz + BT - 1) / BT, 1), BT * N / E, (size_t)N * (BT + 1) * sizeof(C), P->stream>>>(
            S, g, L, (const C*)P->twy, lgT, g.M);
    }
    flups_prof_end(P);
    FLUPS_COUNT(P, tail_col ? 2 : 1);
}

template <typename T, bool INV>
void run_ycol(flups_plan P, typename cplx<T>::t* S, const Geo& g, bool tail_col = true) {
    const int e = e_for<T>(g.ny);
    if (e == 4) run_ycol_e<T, 4, INV>(P, S, g, tail_col);
    else if (e == 8) run_ycol_e<T, 8, INV>(P, S, g, tail_col);
    else if (e == 12) run_ycol_e<T, 12, INV>(P, S, g, tail_col);
    else run_ycol_e<T, Ebig<T>::E, INV>(P, S, g, tail_col);
}

template <typename T, int E>
void run_zper_e(flups_plan P, typename cplx<T>::t* S, const Geo& g, bool tail_col);

template <typename T>
void run_zsolve(flups_plan P, typename cplx<T>::t* S, const Geo& g, bool tail_col = true) {
    typedef typename cplx<T>::t C;
    if (!g.walls) {
        const int e = e_for<T>(g.nz);
        if (e == 4) run_zper_e<T, 4>(P, S, g, tail_col);
        else if (e == 8) run_zper_e<T, 8>(P, S, g, tail_col);
        else if (e == 12) run_zper_e<T, 12>(P, S, g, tail_col);
        else run_zper_e<T, Ebig<T>::E>(P, S, g, tail_col);
    } else {
        const int ncols = g.nxh * g.ny;
        flups_prof_begin(P, sizeof(T) == 4 ? FK_ZTRI32 : FK_ZTRI64);
        if (sizeof(T) == 4 && !g.xpack) {   // tiles in shared memory, no HBM scratch (cols_kernels.cu)
            const int n = launch_ztri_tile(P, (float2*)S, g);
            if (n > 0) {
                flups_prof_end(P);
                FLUPS_COUNT(P, n);
                return;
            }
        }
        if (g.xpack)
            k_ztri_packed<T><<<(ncols + 127) / 128, 128, 0, P->stream>>>(S, (T*)P->zscr, g, (const T*)P->lamx,
                                                                       (const T*)P->lamy, (const T*)P->tri);
        else
            k_ztri<T><<<(ncols + 127) / 128, 128, 0, P->stream>>>(S, (T*)P->zscr, g, (const T*)P->lamx,
                                                                    (const T*)P->lamy, (const T*)P->tri);
        flups_prof_end(P);
        FLUPS_COUNT(P, 1);
    }
}

template <typename T, int E>
void run_zper_e(flups_plan P, typename cplx<T>::t* S, const Geo& g, bool tail_col) {
    typedef typename cplx<T>::t C;
    if (!g.walls) {
        const int N = g.nz;
        const int lgB = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, g.M, g.cta);
        const int B = 1 << lgB;
        const FftLen L = packed(P->lz);
        auto kern = k_zper<T, E, false>;
        auto tail = k_zper<T, E, true>;
        allow_smem(kern);
        allow_smem(tail);
        flups_prof_begin(P, sizeof(T) == 4 ? FK_ZPER32 : FK_ZPER64);
        if (sizeof(T) == 4 && E == 8 && pipe_ok(P, N, 1))
            run_cols_pipe<1, false>(P, (float2*)S, g, L, (const float2*)P->twz);
        else
            kern<<<dim3((g.M + B - 1) / B, g.ny), B * N / E, (size_t)N * (B + 1) * sizeof(C), P->stream>>>(
                S, g, L, (const C*)P->twz, (const T*)P->lamx, (const T*)P->lamy, (const T*)P->lamz, lgB, 0);
        if (tail_col) {
            const int lgT = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, g.ny, g.cta);
            const int BT = 1 << lgT;
            tail<<<dim3((g.ny + BT - 1) / BT, 1), BT * N / E, (size_t)N * (BT + 1) * sizeof(C), P->stream>>>(
                S, g, L, (const C*)P->twz, (const T*)P->lamx, (const T*)P->lamy, (const T*)P->lamz, lgT, g.M);
        }
        flups_prof_end(P);
        FLUPS_COUNT(P, tail_col ? 2 : 1);
    }
}

template <typename T, int E, int MODE, bool STATS>
void run_xfwd_e(flups_plan P, const double* f, const double* p, const Geo& g) {
    typedef typename cplx<T>::t C;
    const int N = g.M, nrows = g.ny * g.nz;
    const bool tiled = MODE >= 2 && xres_tiled(E, E, N, g.ny);
    if constexpr (MODE >= 2 && E == 8 && sizeof(T) == 4) {
        if (tiled) {                       // the z-marching form of the tiled defect
            // its transform tail: the register four-step rows where M is 64, 128 or 256; the
            // shared-memory Stockham passes otherwise
            auto launch = [&](auto kern, size_t xp, const auto* pp) {
                const size_t smem = xres_smem(N) + (size_t)E * xp * sizeof(float2);
                allow_smem(kern, smem);
                const int kz = xres_kz(g.ny, g.nz);
                flups_prof_begin(P, MODE == 3 ? FK_XRES_NORM32 : FK_XFWD_RES32);
                // f's fixed point: written by the first defect (on the binary32 iterate), read by
                // the norm-only passes of the same solve
                long long* fq = nullptr;
                if (P->fq && MODE == 2 && sizeof(*pp) == 4) {
                    cudaMemsetAsync(&P->sc->fq_bad, 0, sizeof(int), P->stream);
                    fq = P->fq;
                    P->fq_live = 1;
                } else if (P->fq && MODE == 3 && P->fq_live) {
                    fq = P->fq;
                }
                kern<<<dim3(g.ny / E, (g.nz + kz - 1) / kz), N, smem, P->stream>>>(
                    f, pp, (float2*)P->spec, g, packed(P->lx), (const float2*)P->twx, (const float2*)P->twxr, kz,
                    P->sc, P->part, fq, &P->sc->fq_pexp);
                flups_prof_end(P);
                FLUPS_COUNT(P, 1);
            };
            auto pick = [&](const auto* pp) {
                typedef typename std::remove_cv<typename std::remove_pointer<decltype(pp)>::type>::type PT;
                if constexpr (MODE == 2) {
                    if (N == 64) return launch(k_xres_zm<E, MODE, 8, 8, PT>, XRow<8, 8>::XP, pp);
                    if (N == 128) return launch(k_xres_zm<E, MODE, 16, 8, PT>, XRow<16, 8>::XP, pp);
                    if (N == 256) return launch(k_xres_zm<E, MODE, 16, 16, PT>, XRow<16, 16>::XP, pp);
                }
                launch(k_xres_zm<E, MODE, 0, 0, PT>, 0, pp);
            };
            // p from the binary32 copy of the first FP32 iterate where the inverse pass left one
            if constexpr (MODE == 2) {
                if (P->p32_live) { pick((const float*)P->p32); return; }
            }
            pick(p);
            return;
        }
    }
    const int lgB = tiled ? 3 : pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, nrows, x_cap(g.cta));
    const int B = 1 << lgB;
    auto kern = k_xfwd<T, E, MODE, STATS>;
    allow_smem(kern);
    flups_prof_begin(P, sizeof(T) == 8 ? FK_XFWD64 : (MODE == 3 ? FK_XRES_NORM32 : (MODE >= 1 ? FK_XFWD_RES32 : FK_XFWD_F32)));
    const int nblk = (nrows + B - 1) / B;
    size_t smem = (size_t)N * (B + 1) * sizeof(C);
    if (tiled && xres_smem(N) > smem) smem = xres_smem(N);
    kern<<<nblk, B * N / E, smem, P->stream>>>(
        f, p, (C*)P->spec, g, packed(P->lx), (const C*)P->twx, (const C*)P->twxr, P->tabs64 + 5 * g.nz, lgB, nrows,
        P->sc, P->part);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
}

template <typename T, int MODE, bool STATS>
void run_xfwd(flups_plan P, const double* f, const double* p, const Geo& g) {
    if (sizeof(T) == 4 && MODE == 0 && xrow4_rows(g.M) > 0) {   // the register four-step rows
        flups_prof_begin(P, FK_XFWD_F32);
        const bool ok = launch_xrow4_fwd(P, f, g, STATS);
        flups_prof_end(P);
        if (ok) { FLUPS_COUNT(P, 1); return; }
    }
    const int e = e_for<T>(g.M);
    if (e == 4) run_xfwd_e<T, 4, MODE, STATS>(P, f, p, g);
    else if (e == 8) run_xfwd_e<T, 8, MODE, STATS>(P, f, p, g);
    else if (e == 12) run_xfwd_e<T, 12, MODE, STATS>(P, f, p, g);
    else run_xfwd_e<T, Ebig<T>::E, MODE, STATS>(P, f, p, g);
}

template <typename T, int E, int ACC, bool MEAN, bool SUBM>
void run_xinv_e(flups_plan P, double* p, const Geo& g) {
    typedef typename cplx<T>::t C;
    const int N = g.M, nrows = g.ny * g.nz;
    const int lgB = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, nrows, x_cap(g.cta));
    const int B = 1 << lgB;
    auto kern = k_xinv<T, E, ACC, MEAN, SUBM>;
    allow_smem(kern);
    flups_prof_begin(P, sizeof(T) == 4 ? (ACC ? FK_XINV_ACC32 : FK_XINV32) : FK_XINV64);
    const int nblk = (nrows + B - 1) / B;
    kern<<<nblk, B * N / E, (size_t)N * (B + 1) * sizeof(C), P->stream>>>(
        (const C*)P->spec, p, g, packed(P->lx), (const C*)P->twx, (const C*)P->twxr, lgB, nrows, P->sc, P->part);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
}

template <typename T, int ACC, bool MEAN, bool SUBM>
void run_xinv(flups_plan P, double* p, const Geo& g) {
    if (sizeof(T) == 4 && xrow4_rows(g.M) > 0) {               // the register four-step rows
        flups_prof_begin(P, ACC ? FK_XINV_ACC32 : FK_XINV32);
        const bool ok = launch_xrow4_inv(P, p, g, ACC ? (SUBM ? 1 : 2) : (MEAN ? 0 : 3));
        flups_prof_end(P);
        if (ok) { FLUPS_COUNT(P, 1); return; }
    }
    const int e = e_for<T>(g.M);
    if (e == 4) run_xinv_e<T, 4, ACC, MEAN, SUBM>(P, p, g);
    else if (e == 8) run_xinv_e<T, 8, ACC, MEAN, SUBM>(P, p, g);
    else if (e == 12) run_xinv_e<T, 12, ACC, MEAN, SUBM>(P, p, g);
    else run_xinv_e<T, Ebig<T>::E, ACC, MEAN, SUBM>(P, p, g);
}

template <typename T, int E, int KIND, bool INV, int ACC>
void run_xdct_e(flups_plan P, const double* fin, double* pout, const Geo& g) {
    typedef typename cplx<T>::t C;
    const int N = g.M, nrows = g.ny * g.nz;
    const int lgB = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, nrows, x_cap(g.cta));
    const int B = 1 << lgB;
    auto kern = k_xdct<T, E, KIND, INV, ACC>;
    allow_smem(kern);
    flups_prof_begin(P, INV ? (sizeof(T) == 4 ? (ACC ? FK_XINV_ACC32 : FK_XINV32) : FK_XINV64)
                             : (sizeof(T) == 4 ? FK_XFWD_F32 : FK_XFWD64));
    // KIND 1, 2: the split twiddles and the quarter-wave table; KIND 3, 4: pre- and post-twiddles
    const C* t1 = KIND >= 3 ? (const C*)P->twqx : (const C*)P->twxr;
    const C* t2 = KIND >= 3 ? (const C*)P->twqx + P->M : (const C*)P->twqx;
    kern<<<(nrows + B - 1) / B, B * N / E, (size_t)N * (B + 1) * sizeof(C), P->stream>>>(
        (C*)P->spec, fin, pout, g, packed(P->lx), (const C*)P->twx, t1, t2, lgB, nrows);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
}

template <typename T, int KIND, bool INV, int ACC>
void run_xdct_k(flups_plan P, const double* fin, double* pout, const Geo& g) {
    if (e_for<T>(g.M) == 4) run_xdct_e<T, 4, KIND, INV, ACC>(P, fin, pout, g);
    else run_xdct_e<T, 8, KIND, INV, ACC>(P, fin, pout, g);
}

template <typename T, bool INV, int ACC>
void run_xdct(flups_plan P, const double* fin, double* pout, const Geo& g) {
    switch (P->bcx) {
        case FLUPS_XY_NEUMANN: run_xdct_k<T, 1, INV, ACC>(P, fin, pout, g); break;
        case FLUPS_XY_DIRICHLET: run_xdct_k<T, 2, INV, ACC>(P, fin, pout, g); break;
        case FLUPS_XY_NEU_DIR: run_xdct_k<T, 3, INV, ACC>(P, fin, pout, g); break;
        default: run_xdct_k<T, 4, INV, ACC>(P, fin, pout, g); break;
    }
}

template <typename T, int E, int KIND, bool INV>
void run_ydct_e(flups_plan P, typename cplx<T>::t* S, const Geo& g, int ncols) {
    typedef typename cplx<T>::t C;
    const int N = g.ny;
    const int lgB = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, ncols, g.cta);
    const int B = 1 << lgB;
    auto kern = k_ydct<T, E, KIND, INV>;
    allow_smem(kern);
    flups_prof_begin(P, sizeof(T) == 4 ? FK_YCOL32 : FK_YCOL64);
    kern<<<dim3((ncols + B - 1) / B, g.nz), B * N / E, (size_t)N * (B + 1) * sizeof(C), P->stream>>>(
        S, g, packed(P->ly), (const C*)P->twy, (const C*)P->twqy, lgB, ncols);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
}

template <typename T, int E, int KIND, bool INV>
void run_ydct4_e(flups_plan P, typename cplx<T>::t* S, const Geo& g, int ncols) {
    typedef typename cplx<T>::t C;
    const int N = g.ny, H = N / 2;
    // B complex columns: 2B sub-columns of H points; threads 2B H / E, shared memory H (2B+1)
    int lgB = pick_lgB(N, sizeof(C), E, sizeof(T) == 4 ? 32 : 16, ncols, g.cta);
    while (lgB > 0 && (long)(2 << lgB) * H / E > 1024) --lgB;
    const int B = 1 << lgB;
    auto kern = k_ydct4<T, E, KIND, INV>;
    allow_smem(kern);
    flups_prof_begin(P, sizeof(T) == 4 ? FK_YCOL32 : FK_YCOL64);
    const C* tq = (const C*)P->twqy;
    kern<<<dim3((ncols + B - 1) / B, g.nz), 2 * B * H / E, (size_t)H * (2 * B + 1) * sizeof(C), P->stream>>>(
        S, g, packed(P->ly2), (const C*)P->twy2, tq, tq + H, lgB, ncols);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
}

template <typename T, bool INV>
void run_ydct(flups_plan P, typename cplx<T>::t* S, const Geo& g, int ncols) {
    const bool e4 = e_for<T>(g.ny) == 4, h4 = e_for<T>(g.ny / 2) == 4;
    switch (P->bcy) {
        case FLUPS_XY_NEUMANN:
            if (e4) run_ydct_e<T, 4, 1, INV>(P, S, g, ncols); else run_ydct_e<T, 8, 1, INV>(P, S, g, ncols);
            break;
        case FLUPS_XY_DIRICHLET:
            if (e4) run_ydct_e<T, 4, 2, INV>(P, S, g, ncols); else run_ydct_e<T, 8, 2, INV>(P, S, g, ncols);
            break;
        case FLUPS_XY_NEU_DIR:
            if (h4) run_ydct4_e<T, 4, 3, INV>(P, S, g, ncols); else run_ydct4_e<T, 8, 3, INV>(P, S, g, ncols);
            break;
        default:
            if (h4) run_ydct4_e<T, 4, 4, INV>(P, S, g, ncols); else run_ydct4_e<T, 8, 4, INV>(P, S, g, ncols);
            break;
    }
}

// The transforms along x and y of a plan with Neumann or Dirichlet ends in x or y: forward
// (INV = false) from the real field f into the spectrum, or backward into p (ACC: p += .).
// Along x the spectrum then holds nx real coefficients per row, so the column passes take nx
// columns and no Nyquist column.
template <typename T>
void r2r_forward(flups_plan P, const double* f, const Geo& g, Geo& gc, int& ncols) {
    typedef typename cplx<T>::t C;
    const bool rx = P->bcx != FLUPS_XY_PERIODIC, ry = P->bcy != FLUPS_XY_PERIODIC;
    gc = g;
    ncols = P->M + 1;
    if (rx) {
        run_xdct<T, false, 0>(P, f, nullptr, g);
        ncols = g.xpack ? P->nx / 2 : P->nx;   // two real x modes per column when packed
        gc.M = ncols;
        gc.nxh = ncols;
    } else {
        run_xfwd<T, 0, false>(P, f, nullptr, g);
    }
    if (ry) run_ydct<T, false>(P, (C*)P->spec, gc, ncols);
    else run_ycol<T, false>(P, (C*)P->spec, gc, !rx);
}

template <typename T, int ACC>
void r2r_backward(flups_plan P, double* p, const Geo& g, const Geo& gc, int ncols) {
    typedef typename cplx<T>::t C;
    const bool rx = P->bcx != FLUPS_XY_PERIODIC, ry = P->bcy != FLUPS_XY_PERIODIC;
    if (ry) run_ydct<T, true>(P, (C*)P->spec, gc, ncols);
    else run_ycol<T, true>(P, (C*)P->spec, gc, !rx);
    if (rx) run_xdct<T, true, ACC>(P, nullptr, p, g);
    else run_xinv<T, ACC, false, false>(P, p, g);
}

// FP64 defect of a plan with Neumann or Dirichlet ends: r = f - mf - L p (p null: r = f - mf),
// with the ghost rules of the ends in x and y (periodic wrap, p_ghost = p for Neumann, -p for
// Dirichlet) and the z coefficients az, cz of the plan; part[b] = block sum of r^2.  With
// pass 0, r and p are not touched and part[b] = block sum of dzf_k f (the volume mean).
__global__ void __launch_bounds__(256) k_res_ends(const double* __restrict__ f, const double* __restrict__ p,
                                                  double* __restrict__ r, Geo g, int bcx, int bcy, double mf,
                                                  int pass, const double* __restrict__ dd,
                                                  double* __restrict__ part) {
    // One row (fixed j, k) per CTA iteration, x across the threads: no 64-bit index division.
    const int nrows = g.ny * g.nz, nx = g.nx;
    double acc = 0.0;
    float acc2 = 0.f;
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int k = row / g.ny, j = row - k * g.ny;
        const double* fr = f + (size_t)row * nx;
        if (pass == 0) {
            const double w = __ldg(g.dzf + k);
            for (int i = threadIdx.x; i < nx; i += blockDim.x) acc = fma(__ldg(fr + i), w, acc);
            continue;
        }
        double* rr = r + (size_t)row * nx;
        if (!p) {
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const double rv = __ldg(fr + i) - mf;
                rr[i] = rv;
                acc = fma(rv, rv, acc);
            }
            continue;
        }
        // neighbour rows (y: periodic wrap or the ghost row itself with sign; z: walls clamp with
        // a zero coefficient, or periodic wrap)
        const double* pr = p + (size_t)row * nx;
        const int js = j - 1, jn = j + 1;
        const bool ys_in = js >= 0, yn_in = jn < g.ny;
        // ghost sign of the low and high faces: +1 Neumann, -1 Dirichlet
        const double ylo = (bcy == FLUPS_XY_DIRICHLET || bcy == FLUPS_XY_DIR_NEU) ? -1.0 : 1.0;
        const double yhi = (bcy == FLUPS_XY_DIRICHLET || bcy == FLUPS_XY_NEU_DIR) ? -1.0 : 1.0;
        const double sgs = ys_in || bcy == FLUPS_XY_PERIODIC ? 1.0 : ylo;
        const double sgn = yn_in || bcy == FLUPS_XY_PERIODIC ? 1.0 : yhi;
        const double* ps = (ys_in || bcy == FLUPS_XY_PERIODIC) ? p + ((size_t)k * g.ny + (ys_in ? js : g.ny - 1)) * nx : pr;
        const double* pn = (yn_in || bcy == FLUPS_XY_PERIODIC) ? p + ((size_t)k * g.ny + (yn_in ? jn : 0)) * nx : pr;
        int km, kp;
        if (g.walls) { km = k > 0 ? k - 1 : 0; kp = k < g.nz - 1 ? k + 1 : g.nz - 1; }
        else { km = k == 0 ? g.nz - 1 : k - 1; kp = k + 1 == g.nz ? 0 : k + 1; }
        const double* pb = p + ((size_t)km * g.ny + j) * nx;
        const double* pt = p + ((size_t)kp * g.ny + j) * nx;
        const double azk = __ldg(g.az + k), czk = __ldg(g.cz + k), dk = __ldg(dd + k);
        const double xlo = (bcx == FLUPS_XY_DIRICHLET || bcx == FLUPS_XY_DIR_NEU) ? -1.0 : 1.0;
        const double xhi = (bcx == FLUPS_XY_DIRICHLET || bcx == FLUPS_XY_NEU_DIR) ? -1.0 : 1.0;
        if (sgs == 1.0 && sgn == 1.0 && g.sx == g.sy) {
            // rows with both y neighbours in place and dx = dy: eight FP64 instructions per
            // point; the stopping test's sum of r^2 in binary32 (r rounded by integer operations)
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const double pc = __ldg(pr + i);
                double pw, pe;
                if (i > 0) pw = __ldg(pr + i - 1);
                else pw = bcx == FLUPS_XY_PERIODIC ? __ldg(pr + nx - 1) : xlo * pc;
                if (i + 1 < nx) pe = __ldg(pr + i + 1);
                else pe = bcx == FLUPS_XY_PERIODIC ? __ldg(pr) : xhi * pc;
                double a = fma(g.sx, (pw + pe) + (__ldg(ps + i) + __ldg(pn + i)), mf);
                a = fma(azk, __ldg(pb + i), a);
                a = fma(czk, __ldg(pt + i), a);
                a = fma(-dk, pc, a);
                const double rv = __ldg(fr + i) - a;
                rr[i] = rv;
                const float rf = d2f_bits(rv);
                acc2 = fmaf(rf, rf, acc2);
            }
            continue;
        }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const double pc = __ldg(pr + i);
            double pw, pe;
            if (i > 0) pw = __ldg(pr + i - 1);
            else pw = bcx == FLUPS_XY_PERIODIC ? __ldg(pr + nx - 1) : xlo * pc;
            if (i + 1 < nx) pe = __ldg(pr + i + 1);
            else pe = bcx == FLUPS_XY_PERIODIC ? __ldg(pr) : xhi * pc;
            // L p + mf = sx (pw + pe) + sy (ps + pn) + az pb + cz pt - dd pc + mf,
            // dd = 2 sx + 2 sy + az + cz (the diagonal of the periodic/wall operator)
            double a = fma(g.sx, pw + pe, mf);
            a = fma(g.sy, sgs * __ldg(ps + i) + sgn * __ldg(pn + i), a);
            a = fma(azk, __ldg(pb + i), a);
            a = fma(czk, __ldg(pt + i), a);
            a = fma(-dk, pc, a);
            const double rv = __ldg(fr + i) - a;
            rr[i] = rv;
            acc = fma(rv, rv, acc);
        }
    }
    // part[3b] = block sum of dzf f (pass 0) or of r^2 in FP64; part[3b+1] = the binary32 sums
    // of r^2 from the fast rows (per thread, added in FP64 across the block)
    block_sum_abc<true, true, false>(acc, acc2, 0.f, part);
}

__global__ void k_add_const(double* __restrict__ a, size_t n, double c) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        a[q] += c;
}

// CTAs of the x passes (one partial sum each) for a complex element of csize bytes; with
// residual != 0, of the FP32 residual pass (which may use the tiled fixed-point layout).
int xfwd_blocks(flups_plan P, int csize, int residual) {
    const int nrows = P->ny * P->nz;
    if (!residual && csize == 8 && xrow4_rows(P->M) > 0) return (nrows + xrow4_rows(P->M) - 1) / xrow4_rows(P->M);
    const int E = P->M % 3 == 0 ? 12 : (P->M >= 8 ? 8 : 4);
    if (residual && csize == 8 && P->uniform_h && xres_tiled(E, E, P->M, P->ny)) {
        const int kz = xres_kz(P->ny, P->nz);
        return (P->ny / 8) * ((P->nz + kz - 1) / kz);
    }
    const int lgB = pick_lgB(P->M, csize, E, csize == 8 ? 32 : 16, nrows, x_cap(P->cta_cap));
    return (nrows + (1 << lgB) - 1) >> lgB;
}

// ------------------------------------------------------------ batched ensemble stages
// One launch per stage of the fixed FP32 + FP64-defect sequence covers every member of an
// ensemble: CTA b takes item b of the stage's work list, own[b] = (member m << 20) | tile
// (one load; the members' tiles are listed member after member).  The stage bodies are those
// of the single-plan kernels: Stockham passes with runtime length (E = 8 or 12 elements per
// thread and 256 threads, so a member's tile width is 256 E / N), the register four-step rows
// for the forward pass of M = 64, the z-marching fixed-point defect where its layout fits, the
// z Thomas solve of one column per thread for walls, and per-member reductions.  A member whose
// defect reached rtol skips every later stage (its done flag, read before anything else).
__device__ __forceinline__ bool batch_skip(const BatchMember* __restrict__ mem, int m) {
    const int* sk = mem[m].g.skip;
    return sk && *(volatile const int*)sk;
}

// The member's descriptor into shared memory (all threads copy; one barrier).
__device__ __forceinline__ const BatchMember& batch_member(const BatchMember* __restrict__ mem, int m) {
    __shared__ __align__(16) BatchMember sD;
    static_assert(sizeof(BatchMember) % 4 == 0, "word copy");
    const int* src = reinterpret_cast<const int*>(mem + m);
    int* dst = reinterpret_cast<int*>(&sD);
    for (int i = threadIdx.x; i < (int)(sizeof(BatchMember) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    return sD;
}

__global__ void k_b_reset(const BatchMember* __restrict__ mem, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    DevScalars* sc = mem[m].sc;
    sc->done = 0;
    sc->fin_count = 0u;
    sc->pexp = 0;
}

// KIND 0: the transform of f with the first pass's partial sums; KIND 1: the defect of the
// member's p with its transform (z-marching fixed point, or the untiled body: fixed point on
// one-spacing grids, else FP64).
template <int KIND>
__global__ void __launch_bounds__(FLUPS_BATCH_THREADS, KIND == 1 ? 2 : 3) k_b_xfwd(const BatchMember* __restrict__ mem,
                                                                                   const unsigned* __restrict__ own,
                                                                                   int n) {
    const unsigned w = __ldg(&own[blockIdx.x]);
    const int m = (int)(w >> 20), tile = (int)(w & 0xFFFFFu);
    if (batch_skip(mem, m)) return;
    const BatchMember& D = batch_member(mem, m);
    const int nrows = D.g.ny * D.g.nz;
    if (KIND == 0) {
        if (D.xr4) xrow4_fwd_body<8, 8, true>(tile, D.f, D.spec, D.g, D.twx, D.twxr, nrows, D.part);
        else if (D.ex == 12)
            xfwd_body<float, 12, 0, true>(tile, D.f, nullptr, D.spec, D.g, D.lx, D.twx, D.twxr, D.dd, D.lgx, nrows,
                                          D.sc, D.part);
        else
            xfwd_body<float, 8, 0, true>(tile, D.f, nullptr, D.spec, D.g, D.lx, D.twx, D.twxr, D.dd, D.lgx, nrows,
                                         D.sc, D.part);
    } else if (D.zm) {
        xres_zm_body<8, 2, 0, 0, double>(tile % D.zbx, tile / D.zbx, D.zg, D.f, D.p, D.spec, D.g, D.lx, D.twx, D.twxr,
                                 D.zkz, D.sc, D.part, tile, nullptr, nullptr);
    } else if (D.dmode == 2) {
        if (D.ex == 12)
            xfwd_body<float, 12, 2, false>(tile, D.f, D.p, D.spec, D.g, D.lx, D.twx, D.twxr, D.dd, D.lgx, nrows,
                                           D.sc, D.part);
        else
            xfwd_body<float, 8, 2, false>(tile, D.f, D.p, D.spec, D.g, D.lx, D.twx, D.twxr, D.dd, D.lgx, nrows,
                                          D.sc, D.part);
    } else {
        if (D.ex == 12)
            xfwd_body<float, 12, 1, false>(tile, D.f, D.p, D.spec, D.g, D.lx, D.twx, D.twxr, D.dd, D.lgx, nrows,
                                           D.sc, D.part);
        else
            xfwd_body<float, 8, 1, false>(tile, D.f, D.p, D.spec, D.g, D.lx, D.twx, D.twxr, D.dd, D.lgx, nrows,
                                          D.sc, D.part);
    }
}

template <bool INV>
__global__ void __launch_bounds__(FLUPS_BATCH_THREADS) k_b_ycol(const BatchMember* __restrict__ mem,
                                                               const unsigned* __restrict__ own, int n) {
    const unsigned w = __ldg(&own[blockIdx.x]);
    const int m = (int)(w >> 20), tile = (int)(w & 0xFFFFFu);
    if (batch_skip(mem, m)) return;
    const BatchMember& D = batch_member(mem, m);
    const int B = 1 << D.lgy, nb = (D.g.M + B - 1) / B;
    if (tile < D.ymain) {
        if (D.ey == 12) ycol_body<float, 12, INV, false>(tile % nb, tile / nb, D.spec, D.g, D.ly, D.twy, D.lgy, 0);
        else ycol_body<float, 8, INV, false>(tile % nb, tile / nb, D.spec, D.g, D.ly, D.twy, D.lgy, 0);
    } else {                                // the Nyquist column kx = M, B planes per tile
        if (D.ey == 12) ycol_body<float, 12, INV, true>(tile - D.ymain, 0, D.spec, D.g, D.ly, D.twy, D.lgy, D.g.M);
        else ycol_body<float, 8, INV, true>(tile - D.ymain, 0, D.spec, D.g, D.ly, D.twy, D.lgy, D.g.M);
    }
}

__global__ void __launch_bounds__(FLUPS_BATCH_THREADS) k_b_z(const BatchMember* __restrict__ mem,
                                                            const unsigned* __restrict__ own, int n) {
    const unsigned w = __ldg(&own[blockIdx.x]);
    const int m = (int)(w >> 20), tile = (int)(w & 0xFFFFFu);
    if (batch_skip(mem, m)) return;
    const BatchMember& D = batch_member(mem, m);
    if (D.g.walls) {                        // one column per thread
        ztri_body<float>(tile, D.spec, D.zscr, D.g, D.lamx, D.lamy, D.tri);
        return;
    }
    const int B = 1 << D.lgz, nb = (D.g.M + B - 1) / B;
    if (tile < D.zmain) {
        if (D.ez == 12)
            zper_body<float, 12, false>(tile % nb, tile / nb, D.spec, D.g, D.lz, D.twz, D.lamx, D.lamy, D.lamz, D.lgz, 0);
        else
            zper_body<float, 8, false>(tile % nb, tile / nb, D.spec, D.g, D.lz, D.twz, D.lamx, D.lamy, D.lamz, D.lgz, 0);
    } else {                                // the Nyquist column kx = M, B values of ky per tile
        if (D.ez == 12)
            zper_body<float, 12, true>(tile - D.zmain, 0, D.spec, D.g, D.lz, D.twz, D.lamx, D.lamy, D.lamz, D.lgz,
                                       D.g.M);
        else
            zper_body<float, 8, true>(tile - D.zmain, 0, D.spec, D.g, D.lz, D.twz, D.lamx, D.lamy, D.lamz, D.lgz,
                                      D.g.M);
    }
}

// KIND 0: p = x with the mean's partial sums; 1: p += x - <p_0>; 2: p += x.
template <int KIND>
__global__ void __launch_bounds__(FLUPS_BATCH_THREADS) k_b_xinv(const BatchMember* __restrict__ mem,
                                                               const unsigned* __restrict__ own, int n) {
    constexpr int ACC = KIND == 0 ? 0 : 1;
    constexpr bool MEAN = KIND == 0, SUBM = KIND == 1;
    const unsigned w = __ldg(&own[blockIdx.x]);
    const int m = (int)(w >> 20), tile = (int)(w & 0xFFFFFu);
    if (batch_skip(mem, m)) return;
    const BatchMember& D = batch_member(mem, m);
    const int nrows = D.g.ny * D.g.nz;
    if (D.ex == 12)
        xinv_body<float, 12, ACC, MEAN, SUBM>(tile, D.spec, D.p, D.g, D.lx, D.twx, D.twxr, D.lgx, nrows, D.sc, D.part);
    else
        xinv_body<float, 8, ACC, MEAN, SUBM>(tile, D.spec, D.p, D.g, D.lx, D.twx, D.twxr, D.lgx, nrows, D.sc, D.part);
}

// One CTA per member: the sums of its x or defect stage's partials.  WHAT 0: mean and norm of
// f; 1: the defect norm and the stopping test (sets done); 2: the mean of the first iterate.
// WHAT 0 and 1 also clear pexp for the inverse pass that follows.
template <int WHAT>
__global__ void __launch_bounds__(FIN_THREADS) k_b_fin(const BatchMember* __restrict__ mem, double thr2) {
    __shared__ double red[3][FIN_THREADS / 32];
    const BatchMember& D = mem[blockIdx.x];
    DevScalars* sc = D.sc;
    if (WHAT == 1 && sc->done) return;
    double a = 0.0, b = 0.0, c = 0.0;
    const int np = WHAT == 1 ? D.td : D.tx;   // partials of the defect stage, or of the x stage
    for (int i = threadIdx.x; i < np; i += FIN_THREADS) {
        a += __ldcg(D.part + 3 * i + 0);
        b += __ldcg(D.part + 3 * i + 1);
        c += __ldcg(D.part + 3 * i + 2);
    }
    fin_block_sum(a, b, c, red);
    if (threadIdx.x == 0) {
        if (WHAT == 0) {
            const double mv = a * D.nrm_w;
            sc->mean_f = mv;
            sc->f2 = b - 2.0 * mv * c + D.npts * mv * mv;
            sc->pexp = 0;
        } else if (WHAT == 1) {
            sc->r2 = b;
            if (b <= thr2 * sc->f2) sc->done = 1;
            sc->pexp = 0;
        } else {
            sc->mean_p = a * D.nrm_w;
        }
    }
}

// Sets the conditional handle h to whether some member has not converged (one CTA).
__global__ void k_b_any(const BatchMember* __restrict__ mem, int n, cudaGraphConditionalHandle h) {
    int act = 0;
    for (int m = threadIdx.x; m < n; m += blockDim.x) act |= !batch_skip(mem, m);
    act = __syncthreads_or(act);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, act ? 1u : 0u);
}

// p = the binary32 first iterate p32 (exact) where the solve ends at its first defect; with done
// set, only once the stopping test has passed (*done != 0), so that a fixed kernel sequence can
// hold the copy.  n2 pairs of points.
__global__ void k_p_from32(const float2* __restrict__ p32, double2* __restrict__ p, size_t n2,
                           const int* __restrict__ done) {
    if (done && !*done) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = p32[i];
        p[i] = make_double2((double)v.x, (double)v.y);
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t launch_solve64(flups_plan P, const double* f, double* p) {
    const Geo g = plan_geo(P);
    run_xfwd<double, 0, false>(P, f, nullptr, g);
    run_ycol<double, false>(P, (double2*)P->spec, g);
    run_zsolve<double>(P, (double2*)P->spec, g);
    run_ycol<double, true>(P, (double2*)P->spec, g);
    run_xinv<double, 0, false, false>(P, p, g);
    return cudaGetLastError();
}

cudaError_t launch_solve64_r2r(flups_plan P, const double* f, double* p) {
    const Geo g = plan_geo(P);
    Geo gc;
    int ncols;
    r2r_forward<double>(P, f, g, gc, ncols);
    run_zsolve<double>(P, (double2*)P->spec, gc, P->bcx == FLUPS_XY_PERIODIC);
    r2r_backward<double, 0>(P, p, g, gc, ncols);
    return cudaGetLastError();
}

int ends_res_blocks(flups_plan P) { return std::min(P->ny * P->nz, 2048); }

cudaError_t launch_ends_residual(flups_plan P, const double* f, const double* p, double* r, double mf, int pass) {
    const Geo g = plan_geo(P);
    flups_prof_begin(P, FK_RES_ENDS);
    k_res_ends<<<ends_res_blocks(P), 256, 0, P->stream>>>(f, p, r, g, P->bcx, P->bcy, mf, pass, P->tabs64 + 5 * g.nz,
                                                          P->part);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
    return cudaGetLastError();
}

// One FP32 solve of L d = r for a plan with ends; p = d (acc = 0) or p += d (acc = 1).
cudaError_t launch_ends_solve32(flups_plan P, const double* r, double* p, int acc) {
    const Geo g = plan_geo(P);
    Geo gc;
    int ncols;
    r2r_forward<float>(P, r, g, gc, ncols);
    run_zsolve<float>(P, (float2*)P->spec, gc, P->bcx == FLUPS_XY_PERIODIC);
    if (acc) r2r_backward<float, 1>(P, p, g, gc, ncols);
    else r2r_backward<float, 0>(P, p, g, gc, ncols);
    return cudaGetLastError();
}

cudaError_t launch_add_const(flups_plan P, double* a, double c) {
    k_add_const<<<1024, 256, 0, P->stream>>>(a, P->npts, c);
    FLUPS_COUNT(P, 1);
    return cudaGetLastError();
}

cudaError_t launch_xfwd32_from_f(flups_plan P, const double* f) {
    const Geo g = plan_geo(P);
    P->p32_live = 0;                       // a new solve: no binary32 iterate yet
    P->fq_live = 0;                        // nor a fixed-point copy of f
    run_xfwd<float, 0, true>(P, f, nullptr, g);
    return cudaGetLastError();
}

cudaError_t launch_finalize_f(flups_plan P) {
    const int nblk = xfwd_blocks(P, 8, 0);
    flups_prof_begin(P, FK_FINALIZE);
    k_finalize<<<fin_grid(nblk), FIN_THREADS, 0, P->stream>>>(P->part, nblk, P->sc, 0,
                                                              1.0 / ((double)P->nx * P->ny * P->sum_dzf),
                                                              (double)P->npts, 0, 0.0, P->fin);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
    return cudaGetLastError();
}

cudaError_t launch_xfwd32_residual(flups_plan P, const double* f, const double* p) {
    const Geo g = plan_geo(P);
    if (P->uniform_h) run_xfwd<float, 2, false>(P, f, p, g);
    else run_xfwd<float, 1, false>(P, f, p, g);
    return cudaGetLastError();
}

cudaError_t launch_p_from32(flups_plan P, double* p, bool cond) {
    if (!P->p32_live) return cudaSuccess;
    k_p_from32<<<8 * 152, 256, 0, P->stream>>>((const float2*)P->p32, reinterpret_cast<double2*>(p), P->npts / 2,
                                              cond ? &P->sc->done : nullptr);
    FLUPS_COUNT(P, 1);
    if (!cond) P->p32_live = 0;
    return cudaGetLastError();
}

bool p32_path(int M, int ny) { return xrow4_rows(M) > 0 && e_for<float>(M) == 8 && xres_tiled(8, 8, M, ny); }

cudaError_t launch_xres_norm32(flups_plan P, const double* f, const double* p) {
    launch_p_from32(P, const_cast<double*>(p), false);   // the norm pass reads the binary64 p
    run_xfwd<float, 3, false>(P, f, p, plan_geo(P));
    return cudaGetLastError();
}

// Stopping tests after the second FP32 solve take the defect norm alone (the fused defect +
// transform pass runs only when another solve follows) on one-spacing grids of 2^24 points or
// more: there the exact fixed-point defect has a norm-only form and the transform it saves
// outweighs one more launch.  Other grids take the fused pass every time.
bool xres_norm_first(flups_plan P) { return P->uniform_h && P->npts >= ((size_t)1 << 24); }

cudaError_t launch_finalize_r(flups_plan P) {
    const int nblk = xfwd_blocks(P, 8, 1);
    flups_prof_begin(P, FK_FINALIZE);
    k_finalize<<<fin_grid(nblk), FIN_THREADS, 0, P->stream>>>(P->part, nblk, P->sc, 1, 0.0, 0.0, 0, 0.0, P->fin);
    flups_prof_end(P);
    FLUPS_COUNT(P, 1);
    return cudaGetLastError();
}

cudaError_t launch_yz_solve32(flups_plan P) {
    const Geo g = plan_geo(P);
    run_ycol<float, false>(P, (float2*)P->spec, g);
    run_zsolve<float>(P, (float2*)P->spec, g);
    run_ycol<float, true>(P, (float2*)P->spec, g);
    return cudaGetLastError();
}

cudaError_t launch_xinv32(flups_plan P, double* p, int mode) {
    const Geo g = plan_geo(P);
    cudaMemsetAsync(&P->sc->pexp, 0, sizeof(int), P->stream);
    if (mode == 4 && !P->p32) mode = 0;
    if (mode == 4) {                       // as 0, the iterate kept in binary32 in P->p32
        flups_prof_begin(P, FK_XINV32);
        const bool ok = launch_xrow4_inv(P, p, g, 4);
        flups_prof_end(P);
        if (!ok) return cudaErrorInvalidValue;
        FLUPS_COUNT(P, 1);
        P->p32_live = 1;
    }
    if (mode == 1 && P->p32_live) {        // as 1, the old iterate read from P->p32
        flups_prof_begin(P, FK_XINV_ACC32);
        const bool ok = launch_xrow4_inv(P, p, g, 5);
        flups_prof_end(P);
        if (!ok) return cudaErrorInvalidValue;
        FLUPS_COUNT(P, 1);
        P->p32_live = 0;
        return cudaGetLastError();
    }
    if (mode == 0 || mode == 4) {          // p = delta, and the volume-weighted mean of p
        if (mode == 0) run_xinv<float, 0, true, false>(P, p, g);
        const int nblk = xfwd_blocks(P, 8, 0);
        flups_prof_begin(P, FK_FINALIZE);
        k_finalize<<<fin_grid(nblk), FIN_THREADS, 0, P->stream>>>(P->part, nblk, P->sc, 2,
                                                                  1.0 / ((double)P->nx * P->ny * P->sum_dzf), 0.0, 0,
                                                                  0.0, P->fin);
        flups_prof_end(P);
        FLUPS_COUNT(P, 1);
    } else if (mode == 1) {                // p += delta - <p_0>
        run_xinv<float, 1, false, true>(P, p, g);
    } else {                               // p += delta
        run_xinv<float, 1, false, false>(P, p, g);
    }
    return cudaGetLastError();
}

int flups_pipe_lgB(int N, int M, int kind) { return pipe_lgB(N, M, kind); }

int flups_default_cta() { return cta_threads(); }

size_t flups_part_blocks_needed(int nx, int ny, int nz) {
    const int M = nx / 2, nrows = ny * nz;
    size_t worst = (size_t)(nrows + 7) / 8;      // the tiled residual pass: 8 rows per CTA
    const int cs[2] = {8, 16};
    const int e1 = M % 3 == 0 ? 12 : (M >= 8 ? 8 : 4);
    const int es[2] = {e1, e1};
    for (int q = 0; q < 2; ++q) {
        for (int cap = 256; cap <= 1024; cap *= 2) {     // every CTA cap a plan may use
            const int lgB = pick_lgB(M, cs[q], es[q], cs[q] == 8 ? 32 : 16, nrows, cap);
            const size_t nb = (size_t)((nrows + (1 << lgB) - 1) >> lgB);
            if (nb > worst) worst = nb;
        }
    }
    return worst;
}

// FP32+refine with a fixed kernel sequence and no host synchronisation: the first FP32
// solve, then (max_iter - 1) rounds of {FP64 defect, norm test, FP32 solve of the defect,
// FP64 update}, then a last defect norm.  Once a norm test passes, the device flag
// sc->done makes every later kernel of the sequence return at once, so the result equals
// the host-driven loop's.  Suitable for stream capture into a CUDA graph.
cudaError_t launch_solve32_fixed(flups_plan P, const double* f, double* p, double rtol, int max_iter) {
    const double thr2 = rtol * rtol;
    const double nrm_w = 1.0 / ((double)P->nx * P->ny * P->sum_dzf);
    cudaMemsetAsync(&P->sc->done, 0, sizeof(int), P->stream);
    P->skip_ptr = nullptr;
    launch_xfwd32_from_f(P, f);
    launch_finalize_f(P);
    launch_yz_solve32(P);
    launch_xinv32(P, p, max_iter >= 2 ? 4 : 0);
    P->skip_ptr = &P->sc->done;
    const int nblk = xfwd_blocks(P, 8, 1);
    auto finalize_r = [&]() {
        k_finalize<<<fin_grid(nblk), FIN_THREADS, 0, P->stream>>>(P->part, nblk, P->sc, 1, nrm_w, 0.0, 1, thr2, P->fin);
        FLUPS_COUNT(P, 1);
    };
    // After the first FP32 solve the defect is ~1e-7 and always feeds a second solve, so its pass
    // is the fused defect + transform.  From the second solve on the defect has usually reached
    // rtol: where xres_norm_first holds, its norm is taken alone first, and the fused pass
    // (skipped once converged) runs only when another solve follows.
    const bool norm_first = xres_norm_first(P);
    for (int it = 1; it <= max_iter; ++it) {
        const bool last = it == max_iter;
        if (norm_first && (it >= 2 || last)) {
            launch_xres_norm32(P, f, p);
            finalize_r();
            if (last) break;
        }
        launch_xfwd32_residual(P, f, p);
        if (!norm_first || it == 1) finalize_r();
        if (last) break;
        if (it == 1) launch_p_from32(P, p, true);    // p from the binary32 iterate if the test passed
        launch_yz_solve32(P);
        launch_xinv32(P, p, it == 1 ? 1 : 2);
    }
    P->skip_ptr = nullptr;
    return cudaGetLastError();
}

extern "C" flups_status flups_selftest_wait_timeout(void* stream, int limit) {
    if (limit < 1 || limit > (1 << 20)) return FLUPS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int* err = nullptr;
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e != cudaSuccess) { flups_note_cuda_error(e); return FLUPS_ENOMEM; }
    int h = 0;
    e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, s>>>(limit, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) { flups_note_cuda_error(e); return FLUPS_ECUDA; }
    return h ? FLUPS_ETIMEOUT : FLUPS_OK;
}

// ------------------------------------------------------------ batched ensemble: host side
bool batch_member_ok(flups_plan P) {
    if (P->prec != FLUPS_FP32_REFINE || P->bcx != FLUPS_XY_PERIODIC || P->bcy != FLUPS_XY_PERIODIC) return false;
    auto len_ok = [](int N) {                 // 8 2^a or 12 2^a, at most 256 E points
        const int E = N % 3 == 0 ? 12 : 8;
        if (N < E || N > 256 * E) return false;
        int q = N % 3 == 0 ? N / 3 : N;
        while (q % 2 == 0) q /= 2;
        return q == 1;
    };
    return len_ok(P->M) && len_ok(P->ny) && (P->bc == FLUPS_BC_WALLS || len_ok(P->nz));
}

void batch_member_fill(flups_plan P, const double* f, double* p, BatchMember* D) {
    std::memset(D, 0, sizeof(*D));
    D->g = plan_geo(P);
    D->g.skip = &P->sc->done;
    D->lx = packed(P->lx);
    D->ly = packed(P->ly);
    D->lz = packed(P->lz);
    D->twx = (const float2*)P->twx;
    D->twxr = (const float2*)P->twxr;
    D->twy = (const float2*)P->twy;
    D->twz = (const float2*)P->twz;
    D->lamx = (const float*)P->lamx;
    D->lamy = (const float*)P->lamy;
    D->lamz = (const float*)P->lamz;
    D->tri = (const float*)P->tri;
    D->spec = (float2*)P->spec;
    D->zscr = (float*)P->zscr;
    D->f = f;
    D->p = p;
    D->sc = P->sc;
    D->part = P->part;
    D->dd = P->tabs64 + 5 * P->nz;
    D->nrm_w = 1.0 / ((double)P->nx * P->ny * P->sum_dzf);
    D->npts = (double)P->npts;
    auto ecls = [](int N) { return N % 3 == 0 ? 12 : 8; };
    auto lgw = [](int N, int E) { return ilog2i(FLUPS_BATCH_THREADS * E / N); };
    D->ex = ecls(P->M);
    D->ey = ecls(P->ny);
    D->ez = P->bc == FLUPS_BC_WALLS ? 8 : ecls(P->nz);
    D->lgx = lgw(P->M, D->ex);
    D->lgy = lgw(P->ny, D->ey);
    D->lgz = P->bc == FLUPS_BC_WALLS ? 0 : lgw(P->nz, D->ez);
    D->dmode = P->uniform_h ? 2 : 1;
    // M = 64: the register four-step rows take the same 32-row tile as the Stockham body (the
    // forward pass from f; the inverse stays on the Stockham body, whose registers set the
    // occupancy of the batched inverse kernel)
    D->xr4 = P->M == 64 && XRow<8, 8>::B == (1 << D->lgx);
    D->smx = (unsigned)std::max<size_t>((size_t)P->M * ((1 << D->lgx) + 1) * sizeof(float2),
                                        D->xr4 ? XRow<8, 8>::SMEM : 0);   // the x stages' largest
    D->smy = (unsigned)((size_t)P->ny * ((1 << D->lgy) + 1) * sizeof(float2));
    D->smz = P->bc == FLUPS_BC_WALLS ? 0u : (unsigned)((size_t)P->nz * ((1 << D->lgz) + 1) * sizeof(float2));
    const int nrows = P->ny * P->nz, bx = 1 << D->lgx, by = 1 << D->lgy, bz = 1 << D->lgz;
    D->tx = (nrows + bx - 1) / bx;
    D->ymain = (P->M + by - 1) / by * P->nz;
    D->ty = D->ymain + (P->nz + by - 1) / by;
    // the z-marching defect where its layout fits: M a multiple of 32 dividing 256, 8 G | ny
    const int G = P->M > 0 && FLUPS_BATCH_THREADS % P->M == 0 ? FLUPS_BATCH_THREADS / P->M : 0;
    D->zm = P->uniform_h && P->M % 32 == 0 && G >= 1 && P->ny % (8 * G) == 0 && P->M <= 256;
    if (D->zm) {
        D->zg = G;
        D->zkz = std::min(8, P->nz);
        D->zbx = P->ny / (8 * G);
        D->td = D->zbx * ((P->nz + D->zkz - 1) / D->zkz);
        D->smd = (unsigned)((size_t)G * xres_smem(P->M));
    } else {
        D->td = D->tx;
        D->smd = D->smx;
    }
    if (P->bc == FLUPS_BC_WALLS) {
        D->zmain = 0;
        D->tz = (P->nxh * P->ny + FLUPS_BATCH_THREADS - 1) / FLUPS_BATCH_THREADS;
    } else {
        D->zmain = (P->M + bz - 1) / bz * P->ny;
        D->tz = D->zmain + (P->ny + bz - 1) / bz;
    }
}

namespace {

void batch_smem_attrs(const BatchLaunch& L) {
    auto smem_attr = [](auto kern, size_t bytes) {
        if (bytes > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    smem_attr(k_b_xfwd<0>, L.smem_x);
    smem_attr(k_b_xfwd<1>, L.smem_d);
    smem_attr(k_b_xinv<0>, L.smem_x);
    smem_attr(k_b_xinv<1>, L.smem_x);
    smem_attr(k_b_xinv<2>, L.smem_x);
    smem_attr(k_b_ycol<false>, L.smem_y);
    smem_attr(k_b_ycol<true>, L.smem_y);
    smem_attr(k_b_z, L.smem_z);
}

// The first FP32 solve and the first defect test (8 kernels).
int batch_first(const BatchLaunch& L, cudaStream_t st, double thr2) {
    const int T = FLUPS_BATCH_THREADS, n = L.n;
    k_b_reset<<<(n + 127) / 128, 128, 0, st>>>(L.mem, n);
    k_b_xfwd<0><<<L.total_x, T, L.smem_x, st>>>(L.mem, L.ox, n);
    k_b_fin<0><<<n, FIN_THREADS, 0, st>>>(L.mem, thr2);
    k_b_ycol<false><<<L.total_y, T, L.smem_y, st>>>(L.mem, L.oy, n);
    k_b_z<<<L.total_z, T, L.smem_z, st>>>(L.mem, L.oz, n);
    k_b_ycol<true><<<L.total_y, T, L.smem_y, st>>>(L.mem, L.oy, n);
    k_b_xinv<0><<<L.total_x, T, L.smem_x, st>>>(L.mem, L.ox, n);
    k_b_fin<2><<<n, FIN_THREADS, 0, st>>>(L.mem, thr2);
    k_b_xfwd<1><<<L.total_d, T, L.smem_d, st>>>(L.mem, L.od, n);
    k_b_fin<1><<<n, FIN_THREADS, 0, st>>>(L.mem, thr2);
    return 10;
}

// One more FP32 solve of the defect (it = 1: with the mean correction) and the next defect test.
int batch_iteration(const BatchLaunch& L, cudaStream_t st, double thr2, int it) {
    const int T = FLUPS_BATCH_THREADS, n = L.n;
    k_b_ycol<false><<<L.total_y, T, L.smem_y, st>>>(L.mem, L.oy, n);
    k_b_z<<<L.total_z, T, L.smem_z, st>>>(L.mem, L.oz, n);
    k_b_ycol<true><<<L.total_y, T, L.smem_y, st>>>(L.mem, L.oy, n);
    if (it == 1) k_b_xinv<1><<<L.total_x, T, L.smem_x, st>>>(L.mem, L.ox, n);
    else k_b_xinv<2><<<L.total_x, T, L.smem_x, st>>>(L.mem, L.ox, n);
    k_b_xfwd<1><<<L.total_d, T, L.smem_d, st>>>(L.mem, L.od, n);
    k_b_fin<1><<<n, FIN_THREADS, 0, st>>>(L.mem, thr2);
    return 6;
}

}  // namespace

int launch_batch_fixed(const BatchLaunch& L, double rtol, int max_iter) {
    batch_smem_attrs(L);
    const double thr2 = rtol * rtol;
    int k = batch_first(L, L.stream, thr2);
    for (int it = 1; it < max_iter; ++it) k += batch_iteration(L, L.stream, thr2, it);
    return cudaGetLastError() == cudaSuccess ? k : -1;
}

int capture_batch_graph(const BatchLaunch& L, cudaStream_t aux, double rtol, int max_iter, cudaGraph_t* out) {
    *out = nullptr;
    batch_smem_attrs(L);
    const double thr2 = rtol * rtol;
    cudaStream_t st = L.stream;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return -1;
    int k = batch_first(L, st, thr2);
    for (int it = 1; it < max_iter && e == cudaSuccess; ++it) {
        // iteration it runs only while some member is active: k_b_any sets the handle, an IF
        // node holds the iteration's kernels (captured on aux into the node's body graph)
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr);
        cudaGraphConditionalHandle h = 0;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) break;
        k_b_any<<<1, 256, 0, st>>>(L.mem, L.n, h);
        ++k;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd);
        if (e != cudaSuccess) break;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
        if (e != cudaSuccess) break;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        k += batch_iteration(L, aux, thr2, it);
        cudaGraph_t bg = nullptr;
        e = cudaStreamEndCapture(aux, &bg);
        if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return -1;
    }
    *out = g;
    return k;
}
