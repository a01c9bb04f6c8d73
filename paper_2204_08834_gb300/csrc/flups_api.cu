// flups_api.cu - the C ABI declared in include/flups.h: plans, workspace, tables, and the
// sequencing of the kernels (FluTAS Sec. 3.3 projection; Sec. 3.3.1 solver step order).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "flups_impl.cuh"

size_t flups_part_blocks_needed(int nx, int ny, int nz);

namespace {

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
// 2^a or 3 * 2^a
bool smooth23(int n) { return pow2(n) || (n % 3 == 0 && pow2(n / 3)); }

// Radix sequence.  n = 2^m: as many radix-8 passes as possible, then a 4 (or 4, 4 / 2).
// n = 3 * 2^m: radix-4 passes, a 2 if m is odd, then the 3 (every radix divides the 12
// elements per thread that such lengths use).
bool make_len(int n, FftLen* L) {
    if (!smooth23(n)) return false;
    L->n = n;
    L->nst = 0;
    if (n % 3 == 0) {
        int m = 0;
        while ((3 << m) < n) ++m;
        for (int i = 0; i < m / 2; ++i) L->rad[L->nst++] = 4;
        if (m % 2) L->rad[L->nst++] = 2;
        L->rad[L->nst++] = 3;
        return L->nst <= FLUPS_MAX_STAGES;
    }
    int m = 0;
    while ((1 << m) < n) ++m;
    int q = m / 3, r = m % 3;
    if (r == 1 && q >= 1) { q -= 1; r = 4; }
    for (int i = 0; i < q; ++i) L->rad[L->nst++] = 8;
    if (r == 2) L->rad[L->nst++] = 4;
    else if (r == 4) { L->rad[L->nst++] = 4; L->rad[L->nst++] = 4; }
    else if (r == 1) L->rad[L->nst++] = 2;
    return L->nst <= FLUPS_MAX_STAGES;
}

// Sizes the kernels support: 2^a >= 8, or 3 * 2^a >= 24 and a multiple of 8 (x and y).
bool size_ok(int n, int lo) {
    if (pow2(n)) return n >= lo;
    return n % 3 == 0 && pow2(n / 3) && n >= 24 && n % 8 == 0;
}

// -4 sin^2(pi k / n) / h^2: the eigenvalues (2 cos(2 pi k/n) - 2)/h^2 without cancellation.
double eig(int k, int n, double h) {
    const double s = std::sin(M_PI * (double)k / (double)n);
    return -4.0 * s * s / (h * h);
}

// Eigenvalue of mode k along a direction of n cells with the given ends: periodic
// -4 sin^2(pi k/n)/h^2; Neumann at both ends -4 sin^2(pi k/(2n))/h^2 (cosine modes);
// Dirichlet at both ends -4 sin^2(pi (k+1)/(2n))/h^2 (sine modes), Sec. 3.3.1.
double eig_bc(int k, int n, double h, int bc) {
    if (bc == FLUPS_XY_PERIODIC) return eig(k, n, h);
    double s;
    if (bc == FLUPS_XY_NEUMANN || bc == FLUPS_XY_DIRICHLET)
        s = std::sin(M_PI * (double)(bc == FLUPS_XY_NEUMANN ? k : k + 1) / (2.0 * (double)n));
    else
        s = std::sin(M_PI * (double)(2 * k + 1) / (4.0 * (double)n));   // mixed ends
    return -4.0 * s * s / (h * h);
}

bool mixed_bc(int bc) { return bc == FLUPS_XY_NEU_DIR || bc == FLUPS_XY_DIR_NEU; }

// pre-twiddles exp(-i pi (4m+1)/(4n)), m < n/2, then post-twiddles exp(-i pi k/n), k < n/2
template <typename T>
void mixed_twiddles(std::vector<T>& out, int n) {
    const int h = n / 2;
    out.resize(4 * (size_t)h);
    for (int m = 0; m < h; ++m) {
        const double a = M_PI * (4.0 * m + 1.0) / (4.0 * n), b = M_PI * (double)m / (double)n;
        out[2 * m] = (T)std::cos(a);
        out[2 * m + 1] = (T)(-std::sin(a));
        out[2 * (h + m)] = (T)std::cos(b);
        out[2 * (h + m) + 1] = (T)(-std::sin(b));
    }
}

// exp(-i pi k/(2n)), k < count (the quarter-wave twiddle of the cosine/sine transforms)
template <typename T>
void quarter_twiddles(std::vector<T>& out, int n, int count) {
    out.resize(2 * (size_t)count);
    for (int m = 0; m < count; ++m) {
        const double a = M_PI * (double)m / (2.0 * (double)n);
        out[2 * m] = (T)std::cos(a);
        out[2 * m + 1] = (T)(-std::sin(a));
    }
}

struct DevAlloc {
    std::vector<void*> ptrs;
    bool ok = true;
    void* get(size_t bytes) {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) { ok = false; return nullptr; }
        ptrs.push_back(p);
        return p;
    }
};

template <typename T>
void twiddles(std::vector<T>& out, int n, int count) {
    out.resize(2 * (size_t)count);
    for (int m = 0; m < count; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)n;
        out[2 * m] = (T)std::cos(a);
        out[2 * m + 1] = (T)(-std::sin(a));
    }
}

template <typename T>
bool upload(void** dst, const std::vector<T>& v, DevAlloc& A) {
    *dst = A.get(v.size() * sizeof(T));
    if (!*dst) return false;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

template <typename T>
bool build_tables(flups_plan P, const std::vector<double>& dzf, DevAlloc& A) {
    std::vector<T> tw;
    twiddles(tw, P->M, P->M);
    if (!upload(&P->twx, tw, A)) return false;
    twiddles(tw, P->nx, P->M / 2 + 1);
    if (!upload(&P->twxr, tw, A)) return false;
    twiddles(tw, P->ny, P->ny);
    if (!upload(&P->twy, tw, A)) return false;
    const bool walls = P->bc == FLUPS_BC_WALLS;
    // inverse of the overall normalisation of the unnormalised transforms
    const double scale = (double)P->M * P->ny * (walls ? 1.0 : (double)P->nz);
    std::vector<T> lx(P->Wx), ly(P->ny);
    for (int k = 0; k < P->Wx; ++k) lx[k] = (T)(eig_bc(k, P->nx, P->dx, P->bcx) * scale);
    for (int k = 0; k < P->ny; ++k) ly[k] = (T)(eig_bc(k, P->ny, P->dy, P->bcy) * scale);
    if (!upload(&P->lamx, lx, A) || !upload(&P->lamy, ly, A)) return false;
    if (P->bcx != FLUPS_XY_PERIODIC) {
        if (mixed_bc(P->bcx)) mixed_twiddles(tw, P->nx);
        else quarter_twiddles(tw, P->nx, P->M + 1);
        if (!upload(&P->twqx, tw, A)) return false;
    }
    if (P->bcy != FLUPS_XY_PERIODIC) {
        if (mixed_bc(P->bcy)) {
            mixed_twiddles(tw, P->ny);
            if (!upload(&P->twqy, tw, A)) return false;
            twiddles(tw, P->ny / 2, P->ny / 2);
            if (!upload(&P->twy2, tw, A)) return false;
        } else {
            quarter_twiddles(tw, P->ny, P->ny);
            if (!upload(&P->twqy, tw, A)) return false;
        }
    }
    if (!walls) {
        twiddles(tw, P->nz, P->nz);
        if (!upload(&P->twz, tw, A)) return false;
        std::vector<T> lz(P->nz);
        for (int k = 0; k < P->nz; ++k) lz[k] = (T)(eig(k, P->nz, dzf[0]) * scale);
        if (!upload(&P->lamz, lz, A)) return false;
    } else {
        const int nz = P->nz;
        std::vector<T> tri(3 * (size_t)nz);
        for (int k = 0; k < nz; ++k) {
            const double a = k > 0 ? 1.0 / (dzf[k] * 0.5 * (dzf[k - 1] + dzf[k])) : 0.0;
            const double c = k < nz - 1 ? 1.0 / (dzf[k] * 0.5 * (dzf[k] + dzf[k + 1])) : 0.0;
            tri[k] = (T)(a * scale);
            tri[nz + k] = (T)(-(a + c) * scale);
            tri[2 * nz + k] = (T)(c * scale);
        }
        if (!upload(&P->tri, tri, A)) return false;
        P->zscr = A.get((size_t)P->Wx * P->ny * nz * sizeof(T));
        if (!P->zscr) return false;
    }
    return true;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    }
    return fn;
}

// 3-D tiled map over the FP32 spectrum [nz][ny][ldS] (8-byte complex elements) with box
// (bx, by, bz); rows of the box land densely in shared memory.
bool make_spec_map(CUtensorMap* m, void* spec, int ldS, int ny, int nz, int bx, int by, int bz) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)ldS, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)ldS * 8, (cuuint64_t)ldS * ny * 8};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, spec, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

flups_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FLUPS_OK;
    flups_note_cuda_error(e);
    if (e == cudaErrorMemoryAllocation) return FLUPS_ENOMEM;
    return FLUPS_ECUDA;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Copies the device scalars to the host; reports (and clears) a device-side wait time-out.
flups_status sync_scalars(flups_plan P) {
    cudaError_t e = cudaMemcpyAsync(P->sc_host, P->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (P->sc_host->err) {
        cudaMemsetAsync(&P->sc->err, 0, sizeof(int), P->stream);
        return FLUPS_ETIMEOUT;
    }
    return FLUPS_OK;
}

}  // namespace

static const char* kKernelNames[FK_COUNT] = {
    "k_rho_tiles", "k_face_coeffs", "k_rhs", "k_correct", "k_xfwd_f32", "k_xfwd_residual32", "k_ycol32",
    "k_zper32", "k_ztri32", "k_xinv32", "k_finalize", "k_xfwd64", "k_ycol64", "k_zper64", "k_ztri64", "k_xinv64",
    "k_res64", "k_rho_finalize", "k_mom_umax", "k_momentum", "k_res_ends", "k_xres_norm32", "k_xinv_acc32",
    "k_vof_rec", "k_vof_flux", "k_vof_update"};

void flups_prof_begin(flups_plan P, int kid) {
    P->prof_open = 0;
    if (!P->prof_on || P->prof_n >= P->prof_cap) return;
    if (cudaEventRecord(P->prof_ev[2 * P->prof_n], P->stream) != cudaSuccess) return;
    P->prof_kid[P->prof_n] = kid;
    P->prof_open = 1;
}

void flups_prof_end(flups_plan P) {
    if (!P->prof_open) return;
    P->prof_open = 0;
    if (cudaEventRecord(P->prof_ev[2 * P->prof_n + 1], P->stream) == cudaSuccess) P->prof_n++;
}

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;
void flups_note_cuda_error(cudaError_t e) { g_last_cuda_error = e; }

Geo plan_geo(flups_plan P) {
    Geo g;
    g.nx = P->nx; g.ny = P->ny; g.nz = P->nz; g.M = P->M; g.nxh = P->nxh; g.ldS = P->ldS;
    g.walls = P->bc == FLUPS_BC_WALLS;
    g.iso = P->uniform_h;
    g.h2e = H2E_NONE;
    if (P->uniform_h) {                          // h = 2^t exactly: frexp gives 0.5 * 2^(t+1)
        int ex = 0;
        if (std::frexp(P->dx, &ex) == 0.5) g.h2e = 2 * (ex - 1);
    }
    g.xpack = P->xpack;
    g.sing00 = (P->bcx == FLUPS_XY_PERIODIC || P->bcx == FLUPS_XY_NEUMANN) &&
               (P->bcy == FLUPS_XY_PERIODIC || P->bcy == FLUPS_XY_NEUMANN);
    g.dx = P->dx; g.dy = P->dy;
    g.sx = 1.0 / (P->dx * P->dx); g.sy = 1.0 / (P->dy * P->dy);
    g.idx = 1.0 / P->dx; g.idy = 1.0 / P->dy;
    g.rx = 32;                                   // largest power of two <= 32 dividing nx
    while (P->nx % g.rx) g.rx >>= 1;
    g.lgrx = g.rx == 32 ? 5 : (g.rx == 16 ? 4 : 3);
    g.tnx = P->nx / g.rx;
    g.tny = P->ny / FLUPS_TY;
    g.tnz = (P->nz + FLUPS_KC - 1) / FLUPS_KC;
    g.trange = P->trange;
    g.skip = P->skip_ptr;
    g.cta = P->cta_cap;
    const int nz = P->nz;
    g.idzf = P->tabs64;
    g.az = P->tabs64 + nz;
    g.cz = P->tabs64 + 2 * nz;
    g.idzc = P->tabs64 + 3 * nz;
    g.dzf = P->tabs64 + 4 * nz;
    return g;
}

extern "C" {

const char* flups_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda_error); }

const char* flups_status_string(int s) {
    switch (s) {
        case FLUPS_OK: return "FLUPS_OK";
        case FLUPS_EINVAL: return "FLUPS_EINVAL: invalid argument";
        case FLUPS_EUNSUPPORTED: return "FLUPS_EUNSUPPORTED: size not supported";
        case FLUPS_ENOMEM: return "FLUPS_ENOMEM: device allocation failed";
        case FLUPS_ECUDA: return "FLUPS_ECUDA: CUDA error";
        case FLUPS_ENONFINITE: return "FLUPS_ENONFINITE: non-finite or invalid value";
        case FLUPS_ENOCONV: return "FLUPS_ENOCONV: refinement did not converge";
        case FLUPS_ESTATE: return "FLUPS_ESTATE: call order violated";
        case FLUPS_ETIMEOUT: return "FLUPS_ETIMEOUT: a bounded device-side wait timed out";
        default: return "unknown flups status";
    }
}

flups_status flups_plan_create(flups_plan* out, int nx, int ny, int nz, double dx, double dy,
                               const double* dzf, int bc, int prec, void* stream) {
    return flups_plan_create_bc(out, nx, ny, nz, dx, dy, dzf, FLUPS_XY_PERIODIC, FLUPS_XY_PERIODIC, bc, prec, stream);
}

flups_status flups_plan_create_bc(flups_plan* out, int nx, int ny, int nz, double dx, double dy,
                                  const double* dzf, int bcx, int bcy, int bc, int prec, void* stream) {
    if (!out) return FLUPS_EINVAL;
    *out = nullptr;
    if (bcx < FLUPS_XY_PERIODIC || bcx > FLUPS_XY_DIR_NEU || bcy < FLUPS_XY_PERIODIC || bcy > FLUPS_XY_DIR_NEU)
        return FLUPS_EINVAL;
    const bool ends = bcx != FLUPS_XY_PERIODIC || bcy != FLUPS_XY_PERIODIC;
    if (!dzf || !(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy)) return FLUPS_EINVAL;
    if (bc != FLUPS_BC_PERIODIC && bc != FLUPS_BC_WALLS) return FLUPS_EINVAL;
    if (prec != FLUPS_FP64 && prec != FLUPS_FP32_REFINE) return FLUPS_EINVAL;
    if (nx <= 0 || ny <= 0 || nz <= 0) return FLUPS_EINVAL;
    if (!size_ok(nx, 8) || !size_ok(ny, 8) || nx > 4096 || ny > 4096) return FLUPS_EUNSUPPORTED;
    if (bc == FLUPS_BC_PERIODIC && (!size_ok(nz, 8) || nz > 4096)) return FLUPS_EUNSUPPORTED;
    if (bc == FLUPS_BC_WALLS && (nz < 2 || nz > 8192)) return FLUPS_EUNSUPPORTED;
    std::vector<double> dz(dzf, dzf + nz);
    double sum = 0.0;
    for (int k = 0; k < nz; ++k) {
        if (!(dz[k] > 0.0) || !std::isfinite(dz[k])) return FLUPS_EINVAL;
        sum += dz[k];
    }
    if (bc == FLUPS_BC_PERIODIC)
        for (int k = 1; k < nz; ++k)
            if (dz[k] != dz[0]) return FLUPS_EINVAL;
    if ((size_t)nx * ny * nz >= (size_t)1 << 31) return FLUPS_EUNSUPPORTED;
    // an FP64 line of n complex values needs n * 2 * 16 bytes of shared memory at the
    // narrowest tile, so FP64 transforms are limited to 2048 points
    if (prec == FLUPS_FP64 && (ny > 2048 || (bc == FLUPS_BC_PERIODIC && nz > 2048))) return FLUPS_EUNSUPPORTED;

    flups_plan P = new (std::nothrow) flups_plan_s();
    if (!P) return FLUPS_ENOMEM;
    P->nx = nx; P->ny = ny; P->nz = nz; P->bc = bc; P->prec = prec;
    P->dx = dx; P->dy = dy;
    P->stream = (cudaStream_t)stream;
    cudaGetDevice(&P->dev);
    P->M = nx / 2;
    P->nxh = nx / 2 + 1;
    P->bcx = bcx;
    P->bcy = bcy;
    P->Wx = bcx == FLUPS_XY_PERIODIC ? P->nxh : nx;
    // all-real spectrum (ends in x and y, walls in z): two real x modes per complex column
    P->xpack = bcx != FLUPS_XY_PERIODIC && bcy != FLUPS_XY_PERIODIC && bc == FLUPS_BC_WALLS;
    const int csize = prec == FLUPS_FP64 ? 16 : 8;
    const int align = 128 / csize;
    P->ldS = (P->Wx + align - 1) / align * align;
    P->npts = (size_t)nx * ny * nz;
    P->nspec = (size_t)P->ldS * ny * nz;
    P->sum_dzf = sum;
    P->dz0 = dz[0];
    P->uniform_h = dx == dy;
    for (int k = 0; k < nz; ++k) P->uniform_h = P->uniform_h && dz[k] == dx;
    if (!make_len(P->M, &P->lx) || !make_len(ny, &P->ly) || (bc == FLUPS_BC_PERIODIC && !make_len(nz, &P->lz)) ||
        (mixed_bc(bcy) && !make_len(ny / 2, &P->ly2))) {
        delete P;
        return FLUPS_EUNSUPPORTED;
    }
    DevAlloc A;
    P->spec = A.get(P->nspec * csize);
    P->bx = (double*)A.get(P->npts * sizeof(double));
    P->by = (double*)A.get(P->npts * sizeof(double));
    P->bz = (double*)A.get(P->npts * sizeof(double));
    {
        int rx = 32;
        while (nx % rx) rx >>= 1;
        P->trange = (long long*)A.get((size_t)(nx / rx) * (ny / FLUPS_TY) * ((nz + FLUPS_KC - 1) / FLUPS_KC) * 2 *
                                      sizeof(long long));
    }
    P->sc = (DevScalars*)A.get(sizeof(DevScalars));
    {
        // partials: 3 per x-pass CTA, 2 per stencil tile (density pass), at least 2048 blocks
        int rx = 32;
        while (nx % rx) rx >>= 1;
        const size_t ntiles = (size_t)(nx / rx) * (ny / FLUPS_TY) * ((nz + FLUPS_KC - 1) / FLUPS_KC);
        P->npart = std::max<size_t>(3 * std::max<size_t>(flups_part_blocks_needed(nx, ny, nz), 2048), 2 * ntiles);
    }
    P->part = (double*)A.get(P->npart * sizeof(double));
    P->fin = (double*)A.get(3 * 256 * sizeof(double));
    P->tabs64 = (double*)A.get(6 * (size_t)nz * sizeof(double));
    if (ends && prec == FLUPS_FP32_REFINE) P->rbuf = (double*)A.get(P->npts * sizeof(double));
    if (!ends && prec == FLUPS_FP32_REFINE && P->uniform_h && p32_path(P->M, ny)) {
        P->p32 = (float*)A.get(P->npts * sizeof(float));
        P->fq = (long long*)A.get(P->npts * sizeof(long long));
    }
    bool ok = A.ok;
    if (ok) {
        std::vector<double> t(6 * (size_t)nz);
        const double sx = 1.0 / (dx * dx), sy = 1.0 / (dy * dy);
        for (int k = 0; k < nz; ++k) {
            double dzc_lo, dzc_hi;
            if (bc == FLUPS_BC_PERIODIC) {
                dzc_lo = dzc_hi = dz[0];
            } else {
                dzc_lo = k > 0 ? 0.5 * (dz[k - 1] + dz[k]) : 0.0;
                dzc_hi = k < nz - 1 ? 0.5 * (dz[k] + dz[k + 1]) : 0.0;
            }
            const double a = dzc_lo > 0.0 ? 1.0 / (dz[k] * dzc_lo) : 0.0;
            const double c = dzc_hi > 0.0 ? 1.0 / (dz[k] * dzc_hi) : 0.0;
            t[k] = 1.0 / dz[k];
            t[nz + k] = a;
            t[2 * nz + k] = c;
            t[3 * nz + k] = dzc_hi > 0.0 ? 1.0 / dzc_hi : 0.0;
            t[4 * nz + k] = dz[k];
            t[5 * nz + k] = 2.0 * sx + 2.0 * sy + a + c;
        }
        ok = cudaMemcpy(P->tabs64, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
        ok = ok && cudaMemset(P->spec, 0, P->nspec * csize) == cudaSuccess;
        ok = ok && cudaMemset(P->sc, 0, sizeof(DevScalars)) == cudaSuccess;
    }
    if (ok) ok = prec == FLUPS_FP64 ? build_tables<double>(P, dz, A) : build_tables<float>(P, dz, A);
    if (ok) ok = cudaMallocHost(&P->sc_host, sizeof(DevScalars)) == cudaSuccess;
    if (!ok) {
        for (void* p : A.ptrs) cudaFree(p);
        if (P->sc_host) cudaFreeHost(P->sc_host);
        delete P;
        cudaGetLastError();
        return FLUPS_ENOMEM;
    }
    P->nallocs = (int)A.ptrs.size();
    P->allocs = (void**)std::malloc(A.ptrs.size() * sizeof(void*));
    if (!P->allocs) {
        for (void* p : A.ptrs) cudaFree(p);
        cudaFreeHost(P->sc_host);
        delete P;
        return FLUPS_ENOMEM;
    }
    for (size_t q = 0; q < A.ptrs.size(); ++q) P->allocs[q] = A.ptrs[q];
    P->total_bytes = P->nspec * csize + 3 * P->npts * sizeof(double) +
                     (bc == FLUPS_BC_WALLS ? (size_t)P->Wx * ny * nz * (csize / 2) : 0);
    P->density_set = 0;
    P->launches = 0;
    P->tma_ok = 0;
    P->skip_ptr = nullptr;
    P->cta_cap = flups_default_cta();
    if (prec == FLUPS_FP32_REFINE && !ends) {
        const int By = 1 << flups_pipe_lgB(ny, P->M, 0);
        // z boxes: the periodic column transform's tile, or the walls Thomas kernel's tile
        const int lw = ztri_tile_lgB(nz);
        const int Bz = bc == FLUPS_BC_WALLS ? (lw >= 0 ? 1 << lw : 0) : 1 << flups_pipe_lgB(nz, P->M, 1);
        P->tma_ok = make_spec_map(&P->tm_y, P->spec, P->ldS, ny, nz, By, ny < 256 ? ny : 256, 1) &&
                    (Bz == 0 || make_spec_map(&P->tm_z, P->spec, P->ldS, ny, nz, Bz, 1, nz < 256 ? nz : 256));
    }
    P->hbuf = nullptr;
    P->hsol = nullptr;
    P->vofbuf = nullptr;
    P->cstream = nullptr;
    for (int q = 0; q < 3; ++q) P->hev[q] = nullptr;
    P->vcbuf = nullptr;
    P->vcs_host = nullptr;
    *out = P;
    return FLUPS_OK;
}

flups_status flups_plan_destroy(flups_plan P) {
    if (!P) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    cudaError_t e = cudaStreamSynchronize(P->stream);
    for (int q = 0; q < P->nallocs; ++q) cudaFree(P->allocs[q]);
    if (P->prof_ev) {
        for (int q = 0; q < 2 * P->prof_cap; ++q) cudaEventDestroy(P->prof_ev[q]);
        std::free(P->prof_ev);
        std::free(P->prof_kid);
    }
    std::free(P->allocs);
    if (P->hbuf) cudaFree(P->hbuf);
    if (P->hsol) cudaFree(P->hsol);
    if (P->vofbuf) cudaFree(P->vofbuf);
    if (P->cstream) {
        cudaStreamSynchronize(P->cstream);
        cudaStreamDestroy(P->cstream);
    }
    for (int q = 0; q < 3; ++q)
        if (P->hev[q]) cudaEventDestroy(P->hev[q]);
    if (P->vcbuf) cudaFree(P->vcbuf);
    if (P->vcs_host) cudaFreeHost(P->vcs_host);
    if (P->sc_host) cudaFreeHost(P->sc_host);
    delete P;
    return cuda_status(e);
}

flups_status flups_set_stream(flups_plan P, void* stream) {
    if (!P) return FLUPS_EINVAL;
    P->stream = (cudaStream_t)stream;
    return FLUPS_OK;
}

size_t flups_workspace_bytes(flups_plan P) { return P ? P->total_bytes : 0; }

unsigned long long flups_launch_count(flups_plan P) { return P ? P->launches : 0ull; }

const char* flups_kernel_name(int id) { return (id >= 0 && id < FK_COUNT) ? kKernelNames[id] : "unknown"; }

flups_status flups_set_profiling(flups_plan P, int on) {
    if (!P) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    if (on && !P->prof_ev) {
        const int cap = 1024;
        P->prof_ev = (cudaEvent_t*)std::calloc(2 * cap, sizeof(cudaEvent_t));
        P->prof_kid = (int*)std::calloc(cap, sizeof(int));
        if (!P->prof_ev || !P->prof_kid) return FLUPS_ENOMEM;
        for (int q = 0; q < 2 * cap; ++q)
            if (cudaEventCreate(&P->prof_ev[q]) != cudaSuccess) return FLUPS_ECUDA;
        P->prof_cap = cap;
    }
    P->prof_on = on ? 1 : 0;
    P->prof_n = 0;
    for (int q = 0; q < FK_COUNT; ++q) { P->prof_ms[q] = 0.0; P->prof_cnt[q] = 0; }
    return FLUPS_OK;
}

flups_status flups_profile_read(flups_plan P, double* ms, long long* n) {
    if (!P || !ms || !n) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int q = 0; q < P->prof_n; ++q) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, P->prof_ev[2 * q], P->prof_ev[2 * q + 1]) == cudaSuccess) {
            P->prof_ms[P->prof_kid[q]] += t;
            P->prof_cnt[P->prof_kid[q]] += 1;
        }
    }
    P->prof_n = 0;
    for (int q = 0; q < FK_COUNT; ++q) {
        ms[q] = P->prof_ms[q];
        n[q] = P->prof_cnt[q];
        P->prof_ms[q] = 0.0;
        P->prof_cnt[q] = 0;
    }
    return FLUPS_OK;
}

// Plans with Neumann or Dirichlet ends in x or y take only the Poisson solve.
bool has_ends(flups_plan P) { return P->bcx != FLUPS_XY_PERIODIC || P->bcy != FLUPS_XY_PERIODIC; }

// Sum of the block partials of the last defect pass (3 per block: FP64 sums, binary32 per-thread
// sums of r^2 from the fast rows, zero), in a
// fixed order on the host (synchronises the plan's stream).
flups_status ends_part_sum(flups_plan P, double* out) {
    const int nb = ends_res_blocks(P);
    std::vector<double> h(3 * (size_t)nb);
    cudaError_t e = cudaMemcpyAsync(h.data(), P->part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_status(e);
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += h[3 * (size_t)b] + h[3 * (size_t)b + 1];
    *out = a;
    return FLUPS_OK;
}

// FP32 solves with FP64 defect correction for a plan with ends: r = f - <f> (singular L) or f,
// then d = L32^-1 r, p += d, r = f - <f> - L p in FP64, until ||r|| <= rtol ||f - <f>||; a
// singular L finally gets p shifted to zero volume-weighted mean.
flups_status ends_refine(flups_plan P, const double* f, double* p, double rtol, int max_iter, flups_info* info) {
    if (max_iter < 1 || max_iter > 64 || !(rtol >= 0.0)) return FLUPS_EINVAL;
    const bool sing = plan_geo(P).sing00 != 0;
    const double vol = (double)P->nx * P->ny * P->sum_dzf;
    double mf = 0.0, f2 = 0.0, r2 = 0.0, s = 0.0;
    flups_status st = FLUPS_OK;
    if (sing) {
        st = cuda_status(launch_ends_residual(P, f, nullptr, nullptr, 0.0, 0));
        if (st == FLUPS_OK) st = ends_part_sum(P, &s);
        if (st != FLUPS_OK) return st;
        mf = s / vol;
    }
    st = cuda_status(launch_ends_residual(P, f, nullptr, P->rbuf, mf, 1));
    if (st == FLUPS_OK) st = ends_part_sum(P, &f2);
    if (st != FLUPS_OK) return st;
    if (!std::isfinite(f2)) return FLUPS_ENONFINITE;
    if (f2 == 0.0) {
        if (info) info->rel_res = 0.0;
        return cuda_status(cudaMemsetAsync(p, 0, P->npts * sizeof(double), P->stream));
    }
    double rel = 1.0;
    for (int it = 1; it <= max_iter; ++it) {
        st = cuda_status(launch_ends_solve32(P, P->rbuf, p, it > 1));
        if (st == FLUPS_OK) st = cuda_status(launch_ends_residual(P, f, p, P->rbuf, mf, 1));
        if (st == FLUPS_OK) st = ends_part_sum(P, &r2);
        if (st != FLUPS_OK) return st;
        rel = std::sqrt(r2 / f2);
        if (info) {
            info->iters = it;
            info->rel_res = rel;
            if (it - 1 < FLUPS_HIST) info->rel_res_hist[it - 1] = rel;
        }
        if (!std::isfinite(rel)) return FLUPS_ENONFINITE;
        if (rel <= rtol) break;
    }
    if (sing) {
        st = cuda_status(launch_ends_residual(P, p, nullptr, nullptr, 0.0, 0));
        if (st == FLUPS_OK) st = ends_part_sum(P, &s);
        if (st == FLUPS_OK) st = cuda_status(launch_add_const(P, p, -s / vol));
        if (st != FLUPS_OK) return st;
    }
    return rel <= rtol ? FLUPS_OK : FLUPS_ENOCONV;
}

flups_status flups_set_density(flups_plan P, const double* rho, double rho0) {
    NvtxRange nvtx_("flups_set_density");
    if (!P || !rho || !aligned16(rho) || std::isnan(rho0)) return FLUPS_EINVAL;
    if (has_ends(P)) return FLUPS_EUNSUPPORTED;
    DeviceGuard dg(P->dev);
    const flups_status st = cuda_status(launch_set_density(P, rho, rho0));
    if (st == FLUPS_OK) P->density_set = 1;
    return st;
}

flups_status flups_plan_sync(flups_plan P) {
    if (!P) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    const flups_status st = sync_scalars(P);
    if (st != FLUPS_OK) return st;
    if (P->sc_host->vof_bad) {           // reported once, then cleared
        cudaMemsetAsync(&P->sc->vof_bad, 0, sizeof(int), P->stream);
        return FLUPS_EINVAL;
    }
    return (P->density_set && P->sc_host->bad_rho) ? FLUPS_ENONFINITE : FLUPS_OK;
}

flups_status flups_get_rho0(flups_plan P, double* rho0_host) {
    if (!P || !rho0_host) return FLUPS_EINVAL;
    if (!P->density_set) return FLUPS_ESTATE;
    DeviceGuard dg(P->dev);
    const flups_status st = sync_scalars(P);
    if (st != FLUPS_OK) return st;
    *rho0_host = P->sc_host->rho0;
    return P->sc_host->bad_rho ? FLUPS_ENONFINITE : FLUPS_OK;
}

flups_status flups_rhs(flups_plan P, const double* u, const double* v, const double* w, const double* p_n,
                       const double* p_nm1, double c1, double c2, double dt, double* f) {
    NvtxRange nvtx_("flups_rhs");
    if (!P || !u || !v || !w || !p_n || !f) return FLUPS_EINVAL;
    if (has_ends(P)) return FLUPS_EUNSUPPORTED;
    if (!aligned16(u) || !aligned16(v) || !aligned16(w) || !aligned16(p_n) || !aligned16(f) ||
        (p_nm1 && !aligned16(p_nm1)))
        return FLUPS_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(c1) || !std::isfinite(c2)) return FLUPS_EINVAL;
    if (f == u || f == v || f == w || f == p_n || f == p_nm1) return FLUPS_EINVAL;
    if (!P->density_set) return FLUPS_ESTATE;
    DeviceGuard dg(P->dev);
    return cuda_status(launch_rhs(P, u, v, w, p_n, p_nm1, c1, c2, dt, f));
}

flups_status flups_correct(flups_plan P, const double* p, const double* p_n, const double* p_nm1, double c1,
                           double c2, double dt, double* u, double* v, double* w) {
    NvtxRange nvtx_("flups_correct");
    if (!P || !p || !p_n || !u || !v || !w) return FLUPS_EINVAL;
    if (has_ends(P)) return FLUPS_EUNSUPPORTED;
    if (!aligned16(p) || !aligned16(p_n) || !aligned16(u) || !aligned16(v) || !aligned16(w) ||
        (p_nm1 && !aligned16(p_nm1)))
        return FLUPS_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(c1) || !std::isfinite(c2)) return FLUPS_EINVAL;
    if (!P->density_set) return FLUPS_ESTATE;
    DeviceGuard dg(P->dev);
    return cuda_status(launch_correct(P, p, p_n, p_nm1, c1, c2, dt, u, v, w));
}

flups_status flups_solve(flups_plan P, const double* f, double* p, double rtol, int max_iter, flups_info* info) {
    NvtxRange nvtx_("flups_solve");
    if (!P || !f || !p || f == p || !aligned16(f) || !aligned16(p)) return FLUPS_EINVAL;
    if (std::isnan(rtol)) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    if (info) {
        info->iters = 0;
        info->rel_res = -1.0;
        for (int q = 0; q < FLUPS_HIST; ++q) info->rel_res_hist[q] = -1.0;
    }
    if (has_ends(P)) {
        if (P->prec == FLUPS_FP64) {   // direct; the residual is not evaluated here
            const flups_status st = cuda_status(launch_solve64_r2r(P, f, p));
            if (st == FLUPS_OK && info) info->iters = 1;
            return st;
        }
        return ends_refine(P, f, p, rtol, max_iter, info);
    }
    if (P->prec == FLUPS_FP64) {
        flups_status st = cuda_status(launch_solve64(P, f, p));
        if (st != FLUPS_OK || !info) return st;
        info->iters = 1;
        if (rtol > 0.0) {
            st = cuda_status(launch_residual64_norm(P, f, p));
            if (st == FLUPS_OK) st = sync_scalars(P);
            if (st != FLUPS_OK) return st;
            const double rr = P->sc_host->f2 > 0.0 ? std::sqrt(P->sc_host->r2 / P->sc_host->f2) : 0.0;
            info->rel_res = rr;
            info->rel_res_hist[0] = rr;
            if (!std::isfinite(rr)) return FLUPS_ENONFINITE;
            if (rr > rtol) return FLUPS_ENOCONV;
        }
        return FLUPS_OK;
    }
    if (max_iter < 1 || max_iter > 64 || !(rtol >= 0.0)) return FLUPS_EINVAL;
    // First FP32 solve on f itself (the initial iterate is p = 0, so the defect is f).
    flups_status st = cuda_status(launch_xfwd32_from_f(P, f));
    if (st == FLUPS_OK) st = cuda_status(launch_finalize_f(P));
    if (st == FLUPS_OK) st = cuda_status(launch_yz_solve32(P));
    if (st == FLUPS_OK) st = cuda_status(launch_xinv32(P, p, max_iter >= 2 ? 4 : 0));
    if (st != FLUPS_OK) return st;
    // a solve that ends at its first defect takes p from the binary32 iterate
    auto finish = [&](flups_status s) {
        const flups_status c = cuda_status(launch_p_from32(P, p, false));
        return s != FLUPS_OK ? s : c;
    };
    double rr = -1.0;
    int it = 1;
    const bool norm_first = xres_norm_first(P);
    for (;; ++it) {
        // FP64 defect r = f - <f> - L p, fused with the forward x transform of r; from the
        // second solve on (where xres_norm_first holds) its norm alone first, the same kernel
        // sequence as the graph-capturable solve.
        const bool alone = norm_first && it >= 2;
        st = cuda_status(alone ? launch_xres_norm32(P, f, p) : launch_xfwd32_residual(P, f, p));
        if (st == FLUPS_OK) st = cuda_status(launch_finalize_r(P));
        if (st == FLUPS_OK) st = sync_scalars(P);
        if (st != FLUPS_OK) return st;
        const double f2 = P->sc_host->f2;
        rr = f2 > 0.0 ? std::sqrt(P->sc_host->r2 / f2) : (P->sc_host->r2 > 0.0 ? INFINITY : 0.0);
        if (info) {
            info->iters = it;
            info->rel_res = rr;
            if (it - 1 < FLUPS_HIST) info->rel_res_hist[it - 1] = rr;
        }
        if (!std::isfinite(rr)) return finish(FLUPS_ENONFINITE);
        if (rr <= rtol) return finish(FLUPS_OK);
        if (it >= max_iter) return finish(FLUPS_ENOCONV);
        // delta = L^-1 r in FP32, p += delta in FP64.
        if (alone) st = cuda_status(launch_xfwd32_residual(P, f, p));
        if (st == FLUPS_OK) st = cuda_status(launch_yz_solve32(P));
        if (st == FLUPS_OK) st = cuda_status(launch_xinv32(P, p, it == 1 ? 1 : 2));
        if (st != FLUPS_OK) return st;
    }
}

flups_status flups_solve_graphable(flups_plan P, const double* f, double* p, double rtol, int max_iter) {
    NvtxRange nvtx_("flups_solve_graphable");
    if (!P || !f || !p || f == p || !aligned16(f) || !aligned16(p)) return FLUPS_EINVAL;
    if (P->prec != FLUPS_FP32_REFINE) return FLUPS_EINVAL;
    if (has_ends(P)) return FLUPS_EUNSUPPORTED;
    if (max_iter < 1 || max_iter > 64 || !(rtol >= 0.0)) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    P->last_max_iter = max_iter;
    return cuda_status(launch_solve32_fixed(P, f, p, rtol, max_iter));
}

flups_status flups_solve_result(flups_plan P, double rtol, flups_info* info) {
    if (!P || !info) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    const flups_status st = sync_scalars(P);
    info->iters = 0;
    info->rel_res = -1.0;
    for (int q = 0; q < FLUPS_HIST; ++q) info->rel_res_hist[q] = -1.0;
    if (st != FLUPS_OK) return st;
    const double f2 = P->sc_host->f2;
    const double rr = f2 > 0.0 ? std::sqrt(P->sc_host->r2 / f2) : (P->sc_host->r2 > 0.0 ? INFINITY : 0.0);
    info->rel_res = rr;
    info->rel_res_hist[0] = rr;
    info->iters = P->last_max_iter;
    if (!std::isfinite(rr)) return FLUPS_ENONFINITE;
    return rr <= rtol ? FLUPS_OK : FLUPS_ENOCONV;
}

flups_status flups_project_host(flups_plan P, double* u, double* v, double* w, const double* rho,
                                const double* p_n, const double* p_nm1, double c1, double c2, double dt,
                                double rtol, int max_iter, double* p_out, flups_info* info) {
    NvtxRange nvtx_("flups_project_host");
    if (!P || !u || !v || !w || !rho || !p_n || !p_out) return FLUPS_EINVAL;
    if (has_ends(P)) return FLUPS_EUNSUPPORTED;
    DeviceGuard dg(P->dev);
    const size_t n = P->npts, b = n * sizeof(double);
    if (!P->hbuf) {
        if (cudaMalloc(&P->hbuf, 8 * b) != cudaSuccess) { cudaGetLastError(); P->hbuf = nullptr; return FLUPS_ENOMEM; }
    }
    if (!P->cstream) {
        cudaError_t e = cudaStreamCreateWithFlags(&P->cstream, cudaStreamNonBlocking);
        for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&P->hev[q], cudaEventDisableTiming);
        if (e != cudaSuccess) {          // leave nothing half made: the next call starts over
            for (int q = 0; q < 3; ++q) {
                if (P->hev[q]) cudaEventDestroy(P->hev[q]);
                P->hev[q] = nullptr;
            }
            if (P->cstream) cudaStreamDestroy(P->cstream);
            P->cstream = nullptr;
            return cuda_status(e);
        }
    }
    double* du = P->hbuf;
    double* dv = du + n;
    double* dw = dv + n;
    double* dr = dw + n;
    double* dpn = dr + n;
    double* dpm = dpn + n;
    double* df = dpm + n;
    double* dp = df + n;
    cudaStream_t s = P->stream, cs = P->cstream;
    // Inputs go over the copy stream, rho first: the density pass runs on the plan stream
    // while u, v, w, p_n, p_nm1 are still in flight.
    cudaError_t e = cudaEventRecord(P->hev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, P->hev[0], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dr, rho, b, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(P->hev[1], cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(du, u, b, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v, b, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dw, w, b, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dpn, p_n, b, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && p_nm1) e = cudaMemcpyAsync(dpm, p_nm1, b, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(P->hev[2], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P->hev[1], 0);
    flups_status st = cuda_status(e);
    if (st == FLUPS_OK) st = flups_set_density(P, dr, 0.0);
    if (st == FLUPS_OK) st = cuda_status(cudaStreamWaitEvent(s, P->hev[2], 0));
    if (st == FLUPS_OK) st = flups_rhs(P, du, dv, dw, dpn, p_nm1 ? dpm : nullptr, c1, c2, dt, df);
    if (st == FLUPS_OK) st = flups_solve(P, df, dp, rtol, max_iter, info);
    // p goes back over the copy stream while the correction runs (both only read p).
    if (st == FLUPS_OK) st = cuda_status(cudaEventRecord(P->hev[0], s));
    if (st == FLUPS_OK) st = cuda_status(cudaStreamWaitEvent(cs, P->hev[0], 0));
    if (st == FLUPS_OK) st = cuda_status(cudaMemcpyAsync(p_out, dp, b, cudaMemcpyDeviceToHost, cs));
    if (st == FLUPS_OK) st = flups_correct(P, dp, dpn, p_nm1 ? dpm : nullptr, c1, c2, dt, du, dv, dw);
    if (st == FLUPS_OK) st = cuda_status(cudaMemcpyAsync(u, du, b, cudaMemcpyDeviceToHost, s));
    if (st == FLUPS_OK) st = cuda_status(cudaMemcpyAsync(v, dv, b, cudaMemcpyDeviceToHost, s));
    if (st == FLUPS_OK) st = cuda_status(cudaMemcpyAsync(w, dw, b, cudaMemcpyDeviceToHost, s));
    // No copy touches the caller's buffers after return, whatever the outcome.
    const cudaError_t e1 = cudaStreamSynchronize(cs);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (st != FLUPS_OK) return st;
    return cuda_status(e1 != cudaSuccess ? e1 : e2);
}

flups_status flups_solve_host(flups_plan P, const double* f, double* p_out, double rtol, int max_iter,
                              flups_info* info) {
    NvtxRange nvtx_("flups_solve_host");
    if (!P || !f || !p_out) return FLUPS_EINVAL;
    DeviceGuard dg(P->dev);
    const size_t n = P->npts, b = n * sizeof(double);
    if (!P->hsol) {
        if (cudaMalloc(&P->hsol, 2 * b) != cudaSuccess) { cudaGetLastError(); P->hsol = nullptr; return FLUPS_ENOMEM; }
    }
    double* df = P->hsol;
    double* dp = df + n;
    cudaStream_t s = P->stream;
    flups_status st = cuda_status(cudaMemcpyAsync(df, f, b, cudaMemcpyHostToDevice, s));
    if (st == FLUPS_OK) st = flups_solve(P, df, dp, rtol, max_iter, info);
    if (st == FLUPS_OK || st == FLUPS_ENOCONV) {
        const flups_status sc = cuda_status(cudaMemcpyAsync(p_out, dp, b, cudaMemcpyDeviceToHost, s));
        if (st == FLUPS_OK) st = sc;
    }
    // No copy touches the caller's buffers after return, whatever the outcome.
    const cudaError_t e = cudaStreamSynchronize(s);
    if (st != FLUPS_OK) return st;
    return cuda_status(e);
}

}  // extern "C"
