// noalloc.cu - flups_solve_fp64_noalloc: the FP64 direct Poisson solve of flups_solve for
// callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a solver embedded as a plug-in inside a host
// application that owns and pre-reserves the whole device memory budget, or code that runs
// under a memory manager which forbids allocations once the run has started.  For them this
// entry point takes its workspace (spectrum, Thomas multipliers, twiddle and eigenvalue
// tables) from one fixed, file-scope device array instead of a plan.  The caller still
// passes the right-hand side f and the output p.
//
// The array is FLUPS_NOALLOC_MAX_BYTES (16 MiB) and, like any __device__ variable, every GPU
// that loads the library holds it until the process exits.  Every call uses the same array
// and leaves its contents behind; nothing in it needs to start at zero, because every
// location a call reads is written earlier in the same call.  Two calls whose work
// overlaps on the GPU (different streams, or different host threads on one device) race on
// the array: serialise them.
#include <cmath>
#include <mutex>

#include "flups_impl.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[FLUPS_NOALLOC_MAX_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch per device, with the id of the context it was looked
// up in: a context that replaced it (cudaDeviceReset, then any runtime call) may place the
// array elsewhere, so a changed id repeats the look-up.
struct ScratchSlot {
    unsigned long long ctx_id;
    void* addr;
};
ScratchSlot g_noalloc_slot[kMaxDevices];

// Id of the current context through the driver entry points (no link to libcuda); 0 when it
// cannot be read or no context is current yet.
unsigned long long current_ctx_id() {
    typedef CUresult (*GetCurrentFn)(CUcontext*);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrentFn)a;
            get_id = (GetIdFn)b;
        }
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Set-up of the current device: the device address of the scratch array, looked up with that
// device current by cudaGetSymbolAddress once per device and context.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    ScratchSlot& slot = g_noalloc_slot[dev];
    const unsigned long long id = current_ctx_id();
    if (!slot.addr || id == 0 || id != slot.ctx_id) {
        void* a = nullptr;
        e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        slot.addr = a;
        slot.ctx_id = current_ctx_id();   // the look-up made the device's context current
    }
    *out = slot.addr;
    return cudaSuccess;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Same radix sequence as a plan uses (radix 8 first, then 4/4 or 4 or 2).
void radix_plan(int n, FftLen* L) {
    int m = 0;
    while ((1 << m) < n) ++m;
    L->n = n;
    L->nst = 0;
    int q = m / 3, r = m % 3;
    if (r == 1 && q >= 1) { q -= 1; r = 4; }
    for (int i = 0; i < q; ++i) L->rad[L->nst++] = 8;
    if (r == 2) L->rad[L->nst++] = 4;
    else if (r == 4) { L->rad[L->nst++] = 4; L->rad[L->nst++] = 4; }
    else if (r == 1) L->rad[L->nst++] = 2;
}

struct NaTables {
    double2 *twx, *twxr, *twy, *twz;
    double *lamx, *lamy, *lamz, *tri, *tabs64;
    int nx, ny, nz, M, nxh, walls;
    double dx, dy, scale;
};

// Twiddles, eigenvalues / normalisation and z coefficients, the same quantities a plan
// computes on the host; tabs64[4nz .. 5nz) already holds dzf.
__global__ void k_noalloc_tables(NaTables t) {
    const int nth = gridDim.x * blockDim.x, tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nz = t.nz;
    const double* dzf = t.tabs64 + 4 * nz;
    for (int m = tid; m < t.M; m += nth) {
        double s, c;
        sincospi(2.0 * m / t.M, &s, &c);
        t.twx[m] = make_double2(c, -s);
    }
    for (int m = tid; m <= t.M / 2; m += nth) {
        double s, c;
        sincospi(2.0 * m / t.nx, &s, &c);
        t.twxr[m] = make_double2(c, -s);
    }
    for (int m = tid; m < t.ny; m += nth) {
        double s, c;
        sincospi(2.0 * m / t.ny, &s, &c);
        t.twy[m] = make_double2(c, -s);
        const double sy = sinpi((double)m / t.ny);
        t.lamy[m] = -4.0 * sy * sy / (t.dy * t.dy) * t.scale;
    }
    for (int k = tid; k < t.nxh; k += nth) {
        const double sx = sinpi((double)k / t.nx);
        t.lamx[k] = -4.0 * sx * sx / (t.dx * t.dx) * t.scale;
    }
    const double sxx = 1.0 / (t.dx * t.dx), syy = 1.0 / (t.dy * t.dy);
    for (int k = tid; k < nz; k += nth) {
        double dzc_lo, dzc_hi;
        if (!t.walls) {
            double s, c;
            sincospi(2.0 * k / nz, &s, &c);
            t.twz[k] = make_double2(c, -s);
            const double sz = sinpi((double)k / nz);
            t.lamz[k] = -4.0 * sz * sz / (dzf[0] * dzf[0]) * t.scale;
            dzc_lo = dzc_hi = dzf[0];
        } else {
            const double a = k > 0 ? 1.0 / (dzf[k] * 0.5 * (dzf[k - 1] + dzf[k])) : 0.0;
            const double c = k < nz - 1 ? 1.0 / (dzf[k] * 0.5 * (dzf[k] + dzf[k + 1])) : 0.0;
            t.tri[k] = a * t.scale;
            t.tri[nz + k] = -(a + c) * t.scale;
            t.tri[2 * nz + k] = c * t.scale;
            dzc_lo = k > 0 ? 0.5 * (dzf[k - 1] + dzf[k]) : 0.0;
            dzc_hi = k < nz - 1 ? 0.5 * (dzf[k] + dzf[k + 1]) : 0.0;
        }
        const double a = dzc_lo > 0.0 ? 1.0 / (dzf[k] * dzc_lo) : 0.0;
        const double c = dzc_hi > 0.0 ? 1.0 / (dzf[k] * dzc_hi) : 0.0;
        t.tabs64[k] = 1.0 / dzf[k];
        t.tabs64[nz + k] = a;
        t.tabs64[2 * nz + k] = c;
        t.tabs64[3 * nz + k] = dzc_hi > 0.0 ? 1.0 / dzc_hi : 0.0;
        t.tabs64[5 * nz + k] = 2.0 * sxx + 2.0 * syy + a + c;
    }
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

flups_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return FLUPS_OK;
    flups_note_cuda_error(e);     // reported by flups_last_cuda_error, as for the plan calls
    return FLUPS_ECUDA;
}

}  // namespace

extern "C" flups_status flups_solve_fp64_noalloc(int nx, int ny, int nz, double dx, double dy, const double* dzf,
                                                 int bc, const double* f, double* p, void* stream) {
    if (!dzf || !f || !p || f == p || ((uintptr_t)f & 15u) || ((uintptr_t)p & 15u)) return FLUPS_EINVAL;
    if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy)) return FLUPS_EINVAL;
    if (bc != FLUPS_BC_PERIODIC && bc != FLUPS_BC_WALLS) return FLUPS_EINVAL;
    if (nx <= 0 || ny <= 0 || nz <= 0) return FLUPS_EINVAL;
    if (!pow2(nx) || !pow2(ny) || nx < 8 || ny < 8 || nx > 4096 || ny > 2048) return FLUPS_EUNSUPPORTED;
    if (bc == FLUPS_BC_PERIODIC && (!pow2(nz) || nz < 8 || nz > 2048)) return FLUPS_EUNSUPPORTED;
    if (bc == FLUPS_BC_WALLS && (nz < 2 || nz > 8192)) return FLUPS_EUNSUPPORTED;
    for (int k = 0; k < nz; ++k) {
        if (!(dzf[k] > 0.0) || !std::isfinite(dzf[k])) return FLUPS_EINVAL;
        if (bc == FLUPS_BC_PERIODIC && dzf[k] != dzf[0]) return FLUPS_EINVAL;
    }
    const bool walls = bc == FLUPS_BC_WALLS;
    const int M = nx / 2, nxh = M + 1, ldS = (nxh + 7) / 8 * 8;

    // Layout of the scratch array for this grid.
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += up256(bytes); return o; };
    const size_t o_tabs = take(6 * (size_t)nz * sizeof(double));
    const size_t o_twx = take((size_t)M * sizeof(double2));
    const size_t o_twxr = take((size_t)(M / 2 + 1) * sizeof(double2));
    const size_t o_twy = take((size_t)ny * sizeof(double2));
    const size_t o_twz = take(walls ? 0 : (size_t)nz * sizeof(double2));
    const size_t o_lamx = take((size_t)nxh * sizeof(double));
    const size_t o_lamy = take((size_t)ny * sizeof(double));
    const size_t o_lamz = take(walls ? 0 : (size_t)nz * sizeof(double));
    const size_t o_tri = take(walls ? 3 * (size_t)nz * sizeof(double) : 0);
    const size_t o_sc = take(sizeof(DevScalars));
    const size_t o_part = take(3 * 64 * sizeof(double));
    const size_t o_spec = take((size_t)ldS * ny * nz * sizeof(double2));
    const size_t o_zscr = take(walls ? (size_t)nxh * ny * nz * sizeof(double) : 0);
    if (off > FLUPS_NOALLOC_MAX_BYTES) return FLUPS_EUNSUPPORTED;

    void* base_v = nullptr;
    cudaError_t e = scratch_address(&base_v);
    if (e != cudaSuccess) return status_of(e);
    unsigned char* base = static_cast<unsigned char*>(base_v);

    // A plan that lives on the host stack and points into the scratch array.
    flups_plan_s P{};
    P.nx = nx; P.ny = ny; P.nz = nz; P.bc = bc; P.prec = FLUPS_FP64;
    cudaGetDevice(&P.dev);
    P.dx = dx; P.dy = dy;
    P.stream = (cudaStream_t)stream;
    P.M = M; P.nxh = nxh; P.ldS = ldS;
    P.npts = (size_t)nx * ny * nz;
    P.nspec = (size_t)ldS * ny * nz;
    radix_plan(M, &P.lx);
    radix_plan(ny, &P.ly);
    if (!walls) radix_plan(nz, &P.lz);
    P.spec = base + o_spec;
    P.zscr = walls ? base + o_zscr : nullptr;
    P.sc = reinterpret_cast<DevScalars*>(base + o_sc);
    P.part = reinterpret_cast<double*>(base + o_part);
    P.npart = 3 * 64;
    P.twx = base + o_twx; P.twxr = base + o_twxr; P.twy = base + o_twy;
    P.twz = walls ? nullptr : base + o_twz;
    P.tabs64 = reinterpret_cast<double*>(base + o_tabs);
    P.lamx = base + o_lamx; P.lamy = base + o_lamy;
    P.lamz = walls ? nullptr : base + o_lamz;
    P.tri = walls ? base + o_tri : nullptr;
    double sum = 0.0;
    for (int k = 0; k < nz; ++k) sum += dzf[k];
    P.sum_dzf = sum;

    e = cudaMemcpyAsync(P.tabs64 + 4 * (size_t)nz, dzf, (size_t)nz * sizeof(double), cudaMemcpyHostToDevice,
                        P.stream);
    if (e != cudaSuccess) return status_of(e);
    NaTables t;
    t.twx = (double2*)P.twx; t.twxr = (double2*)P.twxr; t.twy = (double2*)P.twy; t.twz = (double2*)P.twz;
    t.lamx = (double*)P.lamx; t.lamy = (double*)P.lamy; t.lamz = (double*)P.lamz; t.tri = (double*)P.tri;
    t.tabs64 = P.tabs64;
    t.nx = nx; t.ny = ny; t.nz = nz; t.M = M; t.nxh = nxh; t.walls = walls;
    t.dx = dx; t.dy = dy;
    t.scale = (double)M * ny * (walls ? 1.0 : (double)nz);
    k_noalloc_tables<<<8, 256, 0, P.stream>>>(t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return status_of(e);
    return status_of(launch_solve64(&P, f, p));
}
