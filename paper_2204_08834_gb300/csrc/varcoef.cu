// varcoef.cu - the exact variable-coefficient pressure that the split method approximates.
//
// The split (Sec. 3.3) replaces 1/rho by 1/rho0 and moves the difference to the right-hand
// side through p_hat; with p_hat equal to the exact pressure p_ex of
//     A p = D((rho0/rho_f) G p) = f - <f>_V,   <p>_V = 0,
// the split solve returns p_ex itself.  flups_varcoef_solve computes p_ex by preconditioned
// conjugate gradients in the volume-weighted inner product (a, b) = sum dzf_k a b, in which
// A is symmetric negative semi-definite; the preconditioner is the plan's own constant-
// coefficient solve L^{-1} (L = A at rho = rho0), so the preconditioned operator has its
// spectrum in [rho0/rho_max, 1].  These pressures are the training targets of the learned
// p_hat and the reference of its splitting error.
//
// Workspace (allocated on the first call, owned by the plan; recomputed from rho each call):
// the face coefficients
//   cx = rho0/rho_{i+1/2} / dx^2, cy = rho0/rho_{j+1/2} / dy^2, cz = rho0/rho_{k+1/2} / dzc_k
// (cz = 0 on the top wall face) and the PCG vectors r, z, d, q, all float64 [nz][ny][nx].

#include "flups_impl.cuh"

#include <cmath>

namespace {

constexpr int VC_THREADS = 256;

struct VcScalars {
    double sum;      // last reduction
    double mean;     // volume-weighted mean
    double bb;       // ||f - <f>||^2_w
    double rr;       // ||r||^2_w
    double rz;       // (r, z)_w
    double alpha, beta;
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of v into part[blockIdx.x] (fixed order: deterministic).
__device__ __forceinline__ void block_part(double v, double* part) {
    __shared__ double ws[VC_THREADS / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < VC_THREADS / 32 ? ws[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

struct VcGeo {
    int nx, ny, nz, walls;
    long long n;
    double sx, sy;
    const double* idzf;
    const double* idzc;
    const double* dzf;
};

__global__ void k_vc_coeffs(const double* __restrict__ rho, const DevScalars* __restrict__ sc, VcGeo g,
                            double* __restrict__ cx, double* __restrict__ cy, double* __restrict__ cz) {
    const double r2 = 2.0 * sc->rho0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % g.nx);
        const long long jk = c / g.nx;
        const int j = (int)(jk % g.ny);
        const int k = (int)(jk / g.ny);
        const double rc = rho[c];
        const long long plane = (long long)g.nx * g.ny;
        const double rxp = rho[c - i + (i + 1 == g.nx ? 0 : i + 1)];
        const double ryp = rho[c + (long long)((j + 1 == g.ny ? 0 : j + 1) - j) * g.nx];
        cx[c] = r2 / (rc + rxp) * g.sx;
        cy[c] = r2 / (rc + ryp) * g.sy;
        if (k + 1 == g.nz && g.walls) {
            cz[c] = 0.0;
        } else {
            const double rzp = rho[c + (k + 1 == g.nz ? -(long long)k : 1) * plane];
            cz[c] = r2 / (rc + rzp) * g.idzc[k];
        }
    }
}

// q = A d; part = block partials of (d, q)_w.
__global__ void k_vc_apply(const double* __restrict__ d, double* __restrict__ q, const double* __restrict__ cx,
                           const double* __restrict__ cy, const double* __restrict__ cz, VcGeo g,
                           double* __restrict__ part) {
    double acc = 0.0;
    const long long plane = (long long)g.nx * g.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % g.nx);
        const long long jk = c / g.nx;
        const int j = (int)(jk % g.ny);
        const int k = (int)(jk / g.ny);
        const double dc = d[c];
        const long long xm = c + ((i == 0 ? g.nx : i) - 1 - i);
        const long long xp = c + ((i + 1 == g.nx ? 0 : i + 1) - i);
        const long long ym = c + (long long)((j == 0 ? g.ny : j) - 1 - j) * g.nx;
        const long long yp = c + (long long)((j + 1 == g.ny ? 0 : j + 1) - j) * g.nx;
        double s = cx[c] * (d[xp] - dc) - cx[xm] * (dc - d[xm]) + cy[c] * (d[yp] - dc) - cy[ym] * (dc - d[ym]);
        double sz = 0.0;
        if (!(g.walls && k + 1 == g.nz)) {
            const long long zp = c + (k + 1 == g.nz ? -(long long)k : 1) * plane;
            sz += cz[c] * (d[zp] - dc);
        }
        if (!(g.walls && k == 0)) {
            const long long zm = c + (k == 0 ? (long long)(g.nz - 1) : -1LL) * plane;
            sz -= cz[zm] * (dc - d[zm]);
        }
        s += sz * g.idzf[k];
        q[c] = s;
        acc += g.dzf[k] * dc * s;
    }
    block_part(acc, part);
}

// mode 0: part = (a, 1)_w;  mode 1: r = a - mean, part = (r, r)_w;  mode 2: part = (a, b)_w.
template <int MODE>
__global__ void k_vc_vec(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                         const VcScalars* __restrict__ vs, VcGeo g, double* __restrict__ part) {
    double acc = 0.0;
    const double mean = MODE == 1 ? vs->mean : 0.0;
    const long long plane = (long long)g.nx * g.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.n; c += (long long)gridDim.x * blockDim.x) {
        const double w = g.dzf[c / plane];
        if (MODE == 0) {
            acc += w * a[c];
        } else if (MODE == 1) {
            const double r = a[c] - mean;
            out[c] = r;
            acc += w * r * r;
        } else {
            acc += w * a[c] * b[c];
        }
    }
    block_part(acc, part);
}

// x -= mean, in place.
__global__ void k_vc_shift(double* __restrict__ x, const VcScalars* __restrict__ vs, long long n) {
    const double mean = vs->mean;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        x[c] -= mean;
}

// x += alpha d; r -= alpha q; part = (r, r)_w.
__global__ void k_vc_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ d,
                            const double* __restrict__ q, const VcScalars* __restrict__ vs, VcGeo g,
                            double* __restrict__ part) {
    const double alpha = vs->alpha;
    double acc = 0.0;
    const long long plane = (long long)g.nx * g.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.n; c += (long long)gridDim.x * blockDim.x) {
        x[c] += alpha * d[c];
        const double rn = r[c] - alpha * q[c];
        r[c] = rn;
        acc += g.dzf[c / plane] * rn * rn;
    }
    block_part(acc, part);
}

// d = z + beta d
__global__ void k_vc_dir(double* __restrict__ d, const double* __restrict__ z, const VcScalars* __restrict__ vs,
                         long long n) {
    const double beta = vs->beta;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        d[c] = z[c] + beta * d[c];
}

// Sums the partials in a fixed order and derives the PCG scalars.
// what: 0 mean = S / V; 1 bb = rr = S; 2 rz = S (initial direction); 3 alpha = rz / S;
//       4 rr = S; 5 beta = S / rz, rz = S.
__global__ void k_vc_fin(const double* __restrict__ part, int nblk, VcScalars* vs, int what, double inv_vol) {
    __shared__ double ws[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (int)(blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) {
            vs->sum = s;
            switch (what) {
                case 0: vs->mean = s * inv_vol; break;
                case 1: vs->bb = s; vs->rr = s; break;
                case 2: vs->rz = s; break;
                case 3: vs->alpha = s != 0.0 ? vs->rz / s : 0.0; break;
                case 4: vs->rr = s; break;
                case 5: vs->beta = vs->rz != 0.0 ? s / vs->rz : 0.0; vs->rz = s; break;
            }
        }
    }
}

}  // namespace

struct VcWork {
    double* cx; double* cy; double* cz; double* r; double* z; double* d; double* q;
    double* part;
    VcScalars* vs;
    VcScalars* vs_host;
    int nblk;
};


static VcGeo vc_geo(flups_plan P) {
    const Geo G = plan_geo(P);
    VcGeo g;
    g.nx = P->nx; g.ny = P->ny; g.nz = P->nz; g.walls = P->bc == FLUPS_BC_WALLS;
    g.n = (long long)P->npts;
    g.sx = G.sx; g.sy = G.sy;
    g.idzf = G.idzf; g.idzc = G.idzc; g.dzf = G.dzf;
    return g;
}

// Allocates (once) the PCG workspace of the plan.
static cudaError_t vc_work(flups_plan P, VcWork& W) {
    const size_t n = P->npts;
    int nblk = (int)std::min<size_t>((n + 4 * VC_THREADS - 1) / (4 * VC_THREADS), 1216);
    if (nblk < 1) nblk = 1;
    if (!P->vcbuf) {
        const size_t bytes = 7 * n * sizeof(double) + 2048 * sizeof(double) + sizeof(VcScalars);
        cudaError_t e = cudaMalloc(&P->vcbuf, bytes);
        if (e != cudaSuccess) { P->vcbuf = nullptr; return e; }
        e = cudaMallocHost(&P->vcs_host, sizeof(VcScalars));
        if (e != cudaSuccess) { cudaFree(P->vcbuf); P->vcbuf = nullptr; P->vcs_host = nullptr; return e; }
        P->total_bytes += bytes;
    }
    double* b = (double*)P->vcbuf;
    W.cx = b; W.cy = b + n; W.cz = b + 2 * n; W.r = b + 3 * n; W.z = b + 4 * n; W.d = b + 5 * n; W.q = b + 6 * n;
    W.part = b + 7 * n;
    W.vs = (VcScalars*)(b + 7 * n + 2048);
    W.vs_host = (VcScalars*)P->vcs_host;
    W.nblk = nblk;
    return cudaSuccess;
}

// Preconditioner z = L^{-1} r with the plan's own solve (zero-mean z).
static void vc_precond(flups_plan P, const double* r, double* z) {
    if (P->prec == FLUPS_FP64) launch_solve64(P, r, z);
    else launch_solve32_fixed(P, r, z, 0.0, 3);     // three FP32 passes: FP64-accurate, fixed sequence
}

extern "C" flups_status flups_varcoef_solve(flups_plan P, const double* rho, const double* f, double* p, double rtol,
                                            int max_iter, flups_info* info) {
    NvtxRange nvtx_("flups_varcoef_solve");
    if (!P || !rho || !f || !p || f == p || rho == p) return FLUPS_EINVAL;
    if (((uintptr_t)rho & 15u) || ((uintptr_t)f & 15u) || ((uintptr_t)p & 15u)) return FLUPS_EINVAL;
    if (!(rtol >= 0.0) || max_iter < 1 || max_iter > 100000) return FLUPS_EINVAL;
    if (!P->density_set) return FLUPS_ESTATE;
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != P->dev) cudaSetDevice(P->dev);
    else prev = -1;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};
    if (info) {
        info->iters = 0;
        info->rel_res = -1.0;
        for (int q = 0; q < FLUPS_HIST; ++q) info->rel_res_hist[q] = -1.0;
    }
    VcWork W;
    cudaError_t e = vc_work(P, W);
    if (e != cudaSuccess) { flups_note_cuda_error(e); return e == cudaErrorMemoryAllocation ? FLUPS_ENOMEM : FLUPS_ECUDA; }
    const VcGeo g = vc_geo(P);
    cudaStream_t s = P->stream;
    const int nb = W.nblk;
    const double inv_vol = 1.0 / ((double)P->nx * P->ny * P->sum_dzf);
    k_vc_coeffs<<<nb, VC_THREADS, 0, s>>>(rho, P->sc, g, W.cx, W.cy, W.cz);
    FLUPS_COUNT(P, 1);
    auto fin = [&](int what) { k_vc_fin<<<1, 1024, 0, s>>>(W.part, nb, W.vs, what, inv_vol); FLUPS_COUNT(P, 1); };
    auto sync = [&]() -> flups_status {
        cudaError_t e2 = cudaMemcpyAsync(W.vs_host, W.vs, sizeof(VcScalars), cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        if (e2 != cudaSuccess) { flups_note_cuda_error(e2); return FLUPS_ECUDA; }
        return FLUPS_OK;
    };
    // r = f - <f>, bb = ||r||^2, x = 0
    k_vc_vec<0><<<nb, VC_THREADS, 0, s>>>(f, nullptr, nullptr, W.vs, g, W.part);
    fin(0);
    k_vc_vec<1><<<nb, VC_THREADS, 0, s>>>(f, nullptr, W.r, W.vs, g, W.part);
    fin(1);
    cudaMemsetAsync(p, 0, P->npts * sizeof(double), s);
    FLUPS_COUNT(P, 2);
    flups_status st = sync();
    if (st != FLUPS_OK) return st;
    const double bb = W.vs_host->bb;
    if (!std::isfinite(bb)) return FLUPS_ENONFINITE;
    if (bb == 0.0) {
        if (info) { info->rel_res = 0.0; }
        return FLUPS_OK;
    }
    vc_precond(P, W.r, W.z);
    cudaMemcpyAsync(W.d, W.z, P->npts * sizeof(double), cudaMemcpyDeviceToDevice, s);
    k_vc_vec<2><<<nb, VC_THREADS, 0, s>>>(W.r, W.z, nullptr, W.vs, g, W.part);
    fin(2);
    FLUPS_COUNT(P, 1);
    double rel = 1.0;
    int it = 0;
    while (it < max_iter) {
        ++it;
        k_vc_apply<<<nb, VC_THREADS, 0, s>>>(W.d, W.q, W.cx, W.cy, W.cz, g, W.part);
        fin(3);
        k_vc_update<<<nb, VC_THREADS, 0, s>>>(p, W.r, W.d, W.q, W.vs, g, W.part);
        fin(4);
        FLUPS_COUNT(P, 2);
        st = sync();
        if (st != FLUPS_OK) return st;
        rel = std::sqrt(std::fabs(W.vs_host->rr) / bb);
        if (info) {
            info->iters = it;
            info->rel_res = rel;
            if (it - 1 < FLUPS_HIST) info->rel_res_hist[it - 1] = rel;
        }
        if (!std::isfinite(rel)) return FLUPS_ENONFINITE;
        if (rel <= rtol) break;
        vc_precond(P, W.r, W.z);
        k_vc_vec<2><<<nb, VC_THREADS, 0, s>>>(W.r, W.z, nullptr, W.vs, g, W.part);
        fin(5);
        k_vc_dir<<<nb, VC_THREADS, 0, s>>>(W.d, W.z, W.vs, g.n);
        FLUPS_COUNT(P, 2);
    }
    // p -= <p>_V
    k_vc_vec<0><<<nb, VC_THREADS, 0, s>>>(p, nullptr, nullptr, W.vs, g, W.part);
    fin(0);
    k_vc_shift<<<nb, VC_THREADS, 0, s>>>(p, W.vs, g.n);
    FLUPS_COUNT(P, 2);
    e = cudaGetLastError();
    if (e != cudaSuccess) { flups_note_cuda_error(e); return FLUPS_ECUDA; }
    return rel <= rtol ? FLUPS_OK : FLUPS_ENOCONV;
}
