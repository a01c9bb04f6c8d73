// batch.cu - ensembles of independent FP32-refine Poisson solves of mixed sizes, run as one
// CUDA graph launch.
//
// Every member has its own plan (workspace, tables).  The fixed sequence of the FP32 solve
// with FP64 defect correction (no host synchronisation; a member whose FP64 defect reached
// rtol skips every later stage) runs with one kernel per stage for all members together:
// each stage kernel walks the concatenated (member, tile) list of the ensemble
// (capture_batch_graph, fft_kernels.cu), so the graph holds 7 max_iter + 3 kernels whatever
// the number of members; every iteration after the first sits in a conditional node that
// runs only while some member has not converged.  Ensembles with a member that the stage kernels do not take
// (ends in x or y, lengths other than 8 2^a and 12 2^a) capture each member's own kernel
// sequence instead, round-robin on worker streams forked from the origin stream.  The graph
// is replayed by every later flups_batch_solve with the same arguments.  An optional
// autotuner keeps, per distinct member size, the fastest radix sequence of the power-of-two
// transforms (and, on the per-member path, the CTA thread cap of the transform kernels).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "flups_impl.cuh"

struct flups_batch_s {
    int n = 0, nstreams = 0, dev = 0;
    flups_plan* plans = nullptr;
    cudaStream_t user = nullptr;      // the caller's stream (may be the legacy default stream)
    cudaStream_t origin = nullptr;    // the batch's own stream: captured and launched on
    cudaEvent_t in_ev = nullptr, out_ev = nullptr;
    cudaStream_t* streams = nullptr;
    cudaEvent_t fork = nullptr;
    cudaEvent_t* joins = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const double*> f_cap;
    std::vector<double*> p_cap;
    double rtol_cap = -1.0;
    int maxit_cap = 0;
    unsigned long long graph_kernels = 0;
    std::vector<int> tuned_cta, tuned_radix;
    // the stage kernels' path
    bool staged = false;
    BatchMember* dmem = nullptr;        // device: the members' descriptors
    unsigned* dwork = nullptr;          // device: the stages' work lists
    size_t nwork = 0;
    BatchLaunch bl{};
};

namespace {

// Deterministic pseudo-random right-hand side in [-1, 1] (timing input of the autotuner).
__global__ void k_fill_hash(double* f, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = i + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        f[i] = (double)(long long)(z >> 11) * (1.0 / 4503599627370496.0) - 1.0;
    }
}

// Radix sequence of a power-of-two length: variant 0 = radix-8 passes first (the plan's
// default), variant 1 = radix-4 passes (then a 2).
void radix_variant(FftLen* L, int variant) {
    const int n = L->n;
    if (n % 3 == 0 || variant == 0) return;
    int m = 0;
    while ((1 << m) < n) ++m;
    L->nst = 0;
    for (int i = 0; i < m / 2; ++i) L->rad[L->nst++] = 4;
    if (m % 2) L->rad[L->nst++] = 2;
}

void set_radix(flups_plan P, const FftLen saved[3], int variant) {
    P->lx = saved[0];
    P->ly = saved[1];
    P->lz = saved[2];
    if (variant) {
        radix_variant(&P->lx, 1);
        radix_variant(&P->ly, 1);
        if (P->bc == FLUPS_BC_PERIODIC) radix_variant(&P->lz, 1);
    }
}

flups_status cst(cudaError_t e) {
    if (e != cudaSuccess) flups_note_cuda_error(e);
    return e == cudaSuccess ? FLUPS_OK : (e == cudaErrorMemoryAllocation ? FLUPS_ENOMEM : FLUPS_ECUDA);
}

// Times the graph-capturable solve of one plan for every (CTA cap, radix variant); keeps
// the fastest.  Allocates one temporary f/p pair for the size.
flups_status autotune(flups_plan P, int* best_cta, int* best_radix) {
    const size_t n = P->npts;
    double *f = nullptr, *p = nullptr;
    if (cudaMalloc(&f, n * sizeof(double)) != cudaSuccess) return FLUPS_ENOMEM;
    if (cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) { cudaFree(f); return FLUPS_ENOMEM; }
    k_fill_hash<<<256, 256, 0, P->stream>>>(f, n);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const FftLen saved[3] = {P->lx, P->ly, P->lz};
    float best = 1e30f;
    *best_cta = P->cta_cap;
    *best_radix = 0;
    for (int variant = 0; variant < 2; ++variant) {
        for (int cap = 256; cap <= 1024; cap *= 2) {
            P->cta_cap = cap;
            set_radix(P, saved, variant);
            launch_solve32_fixed(P, f, p, 1e-10, 3);   // warm-up (kernel attributes, caches)
            cudaEventRecord(e0, P->stream);
            for (int r = 0; r < 3; ++r) launch_solve32_fixed(P, f, p, 1e-10, 3);
            cudaEventRecord(e1, P->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (cudaGetLastError() == cudaSuccess && ms < best) {
                best = ms;
                *best_cta = cap;
                *best_radix = variant;
            }
        }
    }
    P->cta_cap = *best_cta;
    set_radix(P, saved, *best_radix);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(f);
    cudaFree(p);
    return cst(cudaGetLastError());
}

// Uploads the members' descriptors and the stages' work lists, and sets B->bl.
cudaError_t staged_setup(flups_batch B, const double* const* f, double* const* p) {
    const int n = B->n;
    std::vector<BatchMember> hm(n);
    std::vector<unsigned> wl[4];
    size_t sx = 0, sy = 0, sz = 0, sd = 0;
    for (int m = 0; m < n; ++m) {
        flups_plan P = B->plans[m];
        batch_member_fill(P, f ? f[m] : nullptr, p ? p[m] : nullptr, &hm[m]);
        const BatchMember& D = hm[m];
        // every stage must cover the member (a member with no defect tiles would read a zero
        // norm); tiles and members must fit the item encoding
        const int t[4] = {D.tx, D.ty, D.tz, D.td};
        for (int q = 0; q < 4; ++q) {
            if (t[q] < 1 || t[q] > (1 << 20) || m >= (1 << 12)) return cudaErrorInvalidValue;
            for (int i = 0; i < t[q]; ++i) wl[q].push_back(((unsigned)m << 20) | (unsigned)i);
        }
        sx = std::max(sx, (size_t)D.smx);
        sy = std::max(sy, (size_t)D.smy);
        sz = std::max(sz, (size_t)D.smz);
        sd = std::max(sd, (size_t)D.smd);
    }
    const size_t tot = wl[0].size() + wl[1].size() + wl[2].size() + wl[3].size();
    if (tot > B->nwork) {
        if (B->dwork) cudaFree(B->dwork);
        B->dwork = nullptr;
        B->nwork = 0;
        cudaError_t e = cudaMalloc(&B->dwork, tot * sizeof(unsigned));
        if (e != cudaSuccess) return e;
        B->nwork = tot;
    }
    cudaError_t e = cudaMemcpy(B->dmem, hm.data(), n * sizeof(BatchMember), cudaMemcpyHostToDevice);
    size_t off = 0;
    const unsigned* base[4];
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
        e = cudaMemcpy(B->dwork + off, wl[q].data(), wl[q].size() * sizeof(unsigned), cudaMemcpyHostToDevice);
        base[q] = B->dwork + off;
        off += wl[q].size();
    }
    if (e != cudaSuccess) return e;
    BatchLaunch& L = B->bl;
    L.mem = B->dmem;
    L.ox = base[0];
    L.oy = base[1];
    L.oz = base[2];
    L.od = base[3];
    L.n = n;
    L.total_x = (int)wl[0].size();
    L.total_y = (int)wl[1].size();
    L.total_z = (int)wl[2].size();
    L.total_d = (int)wl[3].size();
    L.smem_x = sx;
    L.smem_y = sy;
    L.smem_z = sz;
    L.smem_d = sd;
    L.stream = B->origin;
    return e;
}

// Stage-kernel path: per distinct member size, the radix variant whose batched solve of that
// member alone is fastest (timed on the member's own workspace with a seeded right-hand side).
flups_status autotune_staged(flups_batch B, int m) {
    flups_plan P = B->plans[m];
    const size_t n = P->npts;
    double *f = nullptr, *p = nullptr;
    if (cudaMalloc(&f, n * sizeof(double)) != cudaSuccess) return FLUPS_ENOMEM;
    if (cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) { cudaFree(f); return FLUPS_ENOMEM; }
    k_fill_hash<<<256, 256, 0, B->origin>>>(f, n);
    // a one-member view of the batch: the member's plan alone, on the batch's own buffers
    flups_batch_s one;
    one.n = 1;
    one.plans = &B->plans[m];
    one.origin = B->origin;
    one.dmem = B->dmem;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const FftLen saved[3] = {P->lx, P->ly, P->lz};
    float best = 1e30f;
    int bestv = 0;
    for (int variant = 0; variant < 2; ++variant) {
        set_radix(P, saved, variant);
        const double* fa[1] = {f};
        double* pa[1] = {p};
        if (staged_setup(&one, fa, pa) != cudaSuccess) break;
        launch_batch_fixed(one.bl, 1e-10, 3);      // warm-up
        cudaEventRecord(e0, B->origin);
        for (int r = 0; r < 3; ++r) launch_batch_fixed(one.bl, 1e-10, 3);
        cudaEventRecord(e1, B->origin);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (cudaGetLastError() == cudaSuccess && ms < best) { best = ms; bestv = variant; }
    }
    set_radix(P, saved, bestv);
    B->tuned_radix[m] = bestv;
    B->tuned_cta[m] = FLUPS_BATCH_THREADS;
    cudaStreamSynchronize(B->origin);
    if (one.dwork) cudaFree(one.dwork);
    one.plans = nullptr;                // not owned by the view
    one.dmem = nullptr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(f);
    cudaFree(p);
    return cst(cudaGetLastError());
}

void destroy_graph(flups_batch B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
}

flups_status capture(flups_batch B, const double* const* f, double* const* p, double rtol, int max_iter) {
    destroy_graph(B);
    if (B->staged) {
        cudaError_t e = staged_setup(B, f, p);
        if (e != cudaSuccess) return cst(e);
        cudaGraph_t graph = nullptr;
        int k = capture_batch_graph(B->bl, B->streams[0], rtol, max_iter, &graph);
        if (k < 0) {
            // no conditional nodes: the plain sequence (later iterations skip member by member)
            cudaGetLastError();
            e = cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cst(e);
            k = launch_batch_fixed(B->bl, rtol, max_iter);
            e = cudaStreamEndCapture(B->origin, &graph);
            if (e == cudaSuccess && k < 0) e = cudaErrorLaunchFailure;
            if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cst(e); }
        }
        e = cudaGraphInstantiate(&B->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { B->exec = nullptr; return cst(e); }
        for (int m = 0; m < B->n; ++m) B->plans[m]->last_max_iter = max_iter;
        B->graph_kernels = (unsigned long long)k;
        B->f_cap.assign(f, f + B->n);
        B->p_cap.assign(p, p + B->n);
        B->rtol_cap = rtol;
        B->maxit_cap = max_iter;
        return FLUPS_OK;
    }
    cudaError_t e = cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cst(e);
    cudaEventRecord(B->fork, B->origin);
    for (int s = 0; s < B->nstreams; ++s) cudaStreamWaitEvent(B->streams[s], B->fork, 0);
    unsigned long long k0 = 0, k1 = 0;
    for (int m = 0; m < B->n; ++m) k0 += B->plans[m]->launches;
    for (int m = 0; m < B->n; ++m) {
        flups_plan P = B->plans[m];
        P->stream = B->streams[m % B->nstreams];
        launch_solve32_fixed(P, f[m], p[m], rtol, max_iter);
        P->last_max_iter = max_iter;
    }
    for (int m = 0; m < B->n; ++m) k1 += B->plans[m]->launches;
    for (int s = 0; s < B->nstreams; ++s) {
        cudaEventRecord(B->joins[s], B->streams[s]);
        cudaStreamWaitEvent(B->origin, B->joins[s], 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(B->origin, &graph);
    if (e != cudaSuccess) return cst(e);
    e = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { B->exec = nullptr; return cst(e); }
    B->graph_kernels = k1 - k0;
    B->f_cap.assign(f, f + B->n);
    B->p_cap.assign(p, p + B->n);
    B->rtol_cap = rtol;
    B->maxit_cap = max_iter;
    return FLUPS_OK;
}

}  // namespace

extern "C" {

flups_status flups_batch_destroy(flups_batch B) {
    if (!B) return FLUPS_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(B->dev);
    if (B->origin) cudaStreamSynchronize(B->origin);
    destroy_graph(B);
    for (int m = 0; m < B->n; ++m)
        if (B->plans && B->plans[m]) flups_plan_destroy(B->plans[m]);
    for (int s = 0; s < B->nstreams; ++s) {
        if (B->streams && B->streams[s]) cudaStreamDestroy(B->streams[s]);
        if (B->joins && B->joins[s]) cudaEventDestroy(B->joins[s]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->dmem) cudaFree(B->dmem);
    if (B->dwork) cudaFree(B->dwork);
    if (B->in_ev) cudaEventDestroy(B->in_ev);
    if (B->out_ev) cudaEventDestroy(B->out_ev);
    if (B->origin) cudaStreamDestroy(B->origin);
    std::free(B->plans);
    std::free(B->streams);
    std::free(B->joins);
    delete B;
    if (prev >= 0) cudaSetDevice(prev);
    return FLUPS_OK;
}

flups_status flups_batch_create(flups_batch* out, int n, const int* nx, const int* ny, const int* nz,
                                const double* dx, const double* dy, const double* const* dzf, const int* bc,
                                int nstreams, int autotune_on, void* stream) {
    if (!out) return FLUPS_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 4096 || !nx || !ny || !nz || !dx || !dy || !dzf || !bc) return FLUPS_EINVAL;
    if (nstreams < 1) nstreams = 1;
    if (nstreams > 32) nstreams = 32;
    if (nstreams > n) nstreams = n;
    flups_batch B = new (std::nothrow) flups_batch_s();
    if (!B) return FLUPS_ENOMEM;
    cudaGetDevice(&B->dev);
    B->user = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->in_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->out_ev, cudaEventDisableTiming) != cudaSuccess) {
        flups_batch_destroy(B);
        return FLUPS_ECUDA;
    }
    B->plans = (flups_plan*)std::calloc(n, sizeof(flups_plan));
    B->streams = (cudaStream_t*)std::calloc(nstreams, sizeof(cudaStream_t));
    B->joins = (cudaEvent_t*)std::calloc(nstreams, sizeof(cudaEvent_t));
    if (!B->plans || !B->streams || !B->joins) { flups_batch_destroy(B); return FLUPS_ENOMEM; }
    B->nstreams = nstreams;
    for (int s = 0; s < nstreams; ++s) {
        if (cudaStreamCreateWithFlags(&B->streams[s], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->joins[s], cudaEventDisableTiming) != cudaSuccess) {
            flups_batch_destroy(B);
            return FLUPS_ECUDA;
        }
    }
    if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) { flups_batch_destroy(B); return FLUPS_ECUDA; }
    B->n = n;
    for (int m = 0; m < n; ++m) {
        const flups_status st = flups_plan_create(&B->plans[m], nx[m], ny[m], nz[m], dx[m], dy[m], dzf[m], bc[m],
                                                  FLUPS_FP32_REFINE, B->streams[m % nstreams]);
        if (st != FLUPS_OK) { B->n = m; flups_batch_destroy(B); return st; }
    }
    B->tuned_cta.assign(n, B->plans[0]->cta_cap);
    B->tuned_radix.assign(n, 0);
    B->staged = true;
    for (int m = 0; m < n; ++m) B->staged = B->staged && batch_member_ok(B->plans[m]);
    if (B->staged) {
        if (cudaMalloc(&B->dmem, n * sizeof(BatchMember)) != cudaSuccess) {
            flups_batch_destroy(B);
            return FLUPS_ENOMEM;
        }
        B->tuned_cta.assign(n, FLUPS_BATCH_THREADS);
        for (int m = 0; autotune_on && m < n; ++m) {
            int first = -1;   // an earlier member of the same size and boundary condition
            for (int q = 0; q < m && first < 0; ++q)
                if (nx[q] == nx[m] && ny[q] == ny[m] && nz[q] == nz[m] && bc[q] == bc[m]) first = q;
            if (first >= 0) {
                B->plans[m]->lx = B->plans[first]->lx;
                B->plans[m]->ly = B->plans[first]->ly;
                B->plans[m]->lz = B->plans[first]->lz;
                B->tuned_radix[m] = B->tuned_radix[first];
                continue;
            }
            const flups_status st = autotune_staged(B, m);
            if (st != FLUPS_OK) { flups_batch_destroy(B); return st; }
        }
        *out = B;
        return FLUPS_OK;
    }
    if (autotune_on) {
        for (int m = 0; m < n; ++m) {
            int first = -1;   // an earlier member of the same size and boundary condition
            for (int q = 0; q < m && first < 0; ++q)
                if (nx[q] == nx[m] && ny[q] == ny[m] && nz[q] == nz[m] && bc[q] == bc[m]) first = q;
            if (first >= 0) {
                B->plans[m]->cta_cap = B->plans[first]->cta_cap;
                B->plans[m]->lx = B->plans[first]->lx;
                B->plans[m]->ly = B->plans[first]->ly;
                B->plans[m]->lz = B->plans[first]->lz;
                B->tuned_cta[m] = B->tuned_cta[first];
                B->tuned_radix[m] = B->tuned_radix[first];
                continue;
            }
            const flups_status st = autotune(B->plans[m], &B->tuned_cta[m], &B->tuned_radix[m]);
            if (st != FLUPS_OK) { flups_batch_destroy(B); return st; }
        }
    }
    *out = B;
    return FLUPS_OK;
}

flups_status flups_batch_solve(flups_batch B, const double* const* f, double* const* p, double rtol, int max_iter,
                               flups_info* info) {
    NvtxRange nvtx_("flups_batch_solve");
    if (!B || !f || !p || max_iter < 1 || max_iter > 64 || !(rtol >= 0.0)) return FLUPS_EINVAL;
    for (int m = 0; m < B->n; ++m)
        if (!f[m] || !p[m] || f[m] == p[m] || ((uintptr_t)f[m] & 15u) || ((uintptr_t)p[m] & 15u)) return FLUPS_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != B->dev) cudaSetDevice(B->dev);
    bool same = B->exec && rtol == B->rtol_cap && max_iter == B->maxit_cap;
    for (int m = 0; same && m < B->n; ++m) same = f[m] == B->f_cap[m] && p[m] == B->p_cap[m];
    flups_status st = FLUPS_OK;
    if (!same) st = capture(B, f, p, rtol, max_iter);
    // order the graph after the caller's stream, and the caller's stream after the graph
    if (st == FLUPS_OK) st = cst(cudaEventRecord(B->in_ev, B->user));
    if (st == FLUPS_OK) st = cst(cudaStreamWaitEvent(B->origin, B->in_ev, 0));
    if (st == FLUPS_OK) st = cst(cudaGraphLaunch(B->exec, B->origin));
    if (st == FLUPS_OK) st = cst(cudaEventRecord(B->out_ev, B->origin));
    if (st == FLUPS_OK) st = cst(cudaStreamWaitEvent(B->user, B->out_ev, 0));
    if (st == FLUPS_OK && info) {
        st = cst(cudaStreamSynchronize(B->origin));
        for (int m = 0; st == FLUPS_OK && m < B->n; ++m) {
            flups_plan P = B->plans[m];
            cudaError_t e = cudaMemcpy(P->sc_host, P->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { st = cst(e); break; }
            flups_info& I = info[m];
            for (int q = 0; q < FLUPS_HIST; ++q) I.rel_res_hist[q] = -1.0;
            const double f2 = P->sc_host->f2, r2 = P->sc_host->r2;
            I.rel_res = f2 > 0.0 ? std::sqrt(r2 / f2) : (r2 > 0.0 ? INFINITY : 0.0);
            I.rel_res_hist[0] = I.rel_res;
            I.iters = max_iter;
            if (P->sc_host->err) { st = FLUPS_ETIMEOUT; cudaMemset(&P->sc->err, 0, sizeof(int)); }
        }
        if (st == FLUPS_OK)
            for (int m = 0; m < B->n; ++m) {
                if (!std::isfinite(info[m].rel_res)) { st = FLUPS_ENONFINITE; break; }
                if (info[m].rel_res > rtol) st = FLUPS_ENOCONV;
            }
    }
    if (prev >= 0 && prev != B->dev) cudaSetDevice(prev);
    return st;
}

unsigned long long flups_batch_graph_kernels(flups_batch B) { return B ? B->graph_kernels : 0ull; }

flups_status flups_batch_member_tuning(flups_batch B, int m, int* cta_threads, int* radix_variant) {
    if (!B || m < 0 || m >= B->n || !cta_threads || !radix_variant) return FLUPS_EINVAL;
    *cta_threads = B->tuned_cta[m];
    *radix_variant = B->tuned_radix[m];
    return FLUPS_OK;
}

}  // extern "C"
