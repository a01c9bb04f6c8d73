// flups_impl.cuh - internal declarations shared by the CUDA translation units of libflups.
//
// Data layout in HBM (per plan):
//   fields          float64 [nz][ny][nx], caller-owned
//   spectrum S      complex (float2 in FP32-refine mode, double2 in FP64 mode)
//                   [nz][ny][ldS], ldS = nx/2+1 rounded up so every row starts on a
//                   128-byte boundary; entries nx/2+1 .. ldS-1 are never read
//   face coeffs     float64 bx, by, bz [nz][ny][nx]: (1 - rho0/rho_f)/h for the face above
//                   each cell in x, y, z (h = dx, dy, dzc_k); bz = 0 on the top wall face
//   z scratch       T [nz][ny][nx/2+1]: forward-sweep multipliers of the z Thomas solve
//   tables          FP64/FP32 twiddles, eigenvalues, z coefficients
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/flups.h"
#include <nvtx3/nvToolsExt.h>

// One NVTX range per public call, named after it, so that a profiler can attribute kernels to
// calls (for instance `ncu --nvtx --nvtx-include "flups_solve/"`); with no tool attached the
// push and the pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

#define FLUPS_MAX_STAGES 14

// v mod n for v in [-n, 2n): the periodic wrap of a neighbour index (any n, not only 2^k).
__device__ __forceinline__ int wrapm(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <typename T> struct cplx;
template <> struct cplx<float> { typedef float2 t; };
template <> struct cplx<double> { typedef double2 t; };

// One 1-D transform length and its radix sequence (each radix 2, 3, 4 or 8).
struct FftLen {
    int n;
    int nst;
    int rad[FLUPS_MAX_STAGES];
    unsigned long long code;     // rad[] packed 4 bits per stage (filled by the launchers)
};

// Device-side scalars written by the reduction kernels.
struct DevScalars {
    double rho0;        // minimum density
    double inv_rho0;    // 1/rho0
    double m2r0;        // -2 rho0
    double m2r0_dx;     // -2 rho0 / dx
    double m2r0_dy;     // -2 rho0 / dy
    double mean_f;      // volume-weighted mean of f
    double f2;          // ||f - <f>||^2
    double r2;          // ||r||^2 of the last residual pass
    double mean_p;      // volume-weighted mean of the first FP32 iterate p_0
    int    bad_rho;     // nonzero: non-finite, non-positive or out-of-range density seen
    int    pexp;        // largest binary64 exponent field of p written by the last FP32 inverse-x pass
    int    err;         // nonzero: a bounded device-side wait timed out (the result is invalid)
    int    done;        // graph-capturable solve: the defect reached rtol, later iterations skip
    unsigned int fin_count;   // blocks of the running final reduction that have finished
    unsigned int mom_hmax;    // momentum predictor: high word of max(|u|, |v|, |w|)
    int    vof_bad;     // VoF step: a face had |u| dt / h above 1 (or not finite)
    int    fq_pexp;     // scale (pexp) of the fixed-point F - MF written by the first defect (-1: none)
    int    fq_bad;      // nonzero: some point of that F - MF could not be formed
};

// Geometry and tables handed to kernels by value.
// Stencil tiles: a CTA of the rhs/correct kernels covers RX x FLUPS_TY cells of a plane,
// RX = min(32, nx), and marches up FLUPS_KC planes.  set_density records each tile's density
// range over its cells and one-cell halo; a tile whose range is [rho0, rho0] reads only zero
// face coefficients (1 - rho0/rho_f) and takes the constant-density path.
#define FLUPS_TY 8
#define FLUPS_KC 16

#define H2E_NONE (-100000)

struct Geo {
    int nx, ny, nz, M, nxh, ldS, walls, iso;   // iso: dx == dy == every dzf
    int sing00;                  // the (kx, ky) = (0, 0) z column is singular (no Dirichlet end in x, y)
    int h2e;                     // iso with h = 2^t: 2t (h^2 = 2^h2e), else H2E_NONE
    int xpack;                   // x coefficients real and packed two per complex column: X_k is the k-th
                                 // real of the spectrum row (ends in x and y, z walls)
    double dx, dy;
    double idx, idy;             // 1/dx, 1/dy
    double sx, sy;               // 1/dx^2, 1/dy^2
    int rx, lgrx, tnx, tny, tnz; // stencil tile width (a power of two), its log2, tile counts
    const long long* trange;     // [tnz][tny][tnx][2] density range (bit patterns) of each tile and its halo
    const int* skip;             // refinement kernels return at once when *skip != 0 (may be null)
    int cta;                     // thread cap of the transform CTAs (0: library default)
    const double* idzf;          // [nz] 1/dzf_k
    const double* az;            // [nz] Laplacian z sub-diagonal   1/(dzf_k dzc_{k-1}) (0 at k=0 with walls)
    const double* cz;            // [nz] Laplacian z super-diagonal 1/(dzf_k dzc_k) (0 at k=nz-1 with walls)
    const double* idzc;          // [nz] 1/dzc_k (0 on the top wall face)
    const double* dzf;           // [nz]
};

// Optional per-kernel timing (flups_set_profiling): each launcher brackets its kernel(s)
// with CUDA events on the plan's stream.  Kernel ids name the timed regions.
enum FlupsKernelId {
    FK_RHO_MINMAX = 0, FK_FACE_COEFFS, FK_RHS, FK_CORRECT, FK_XFWD_F32, FK_XFWD_RES32, FK_YCOL32, FK_ZPER32,
    FK_ZTRI32, FK_XINV32, FK_FINALIZE, FK_XFWD64, FK_YCOL64, FK_ZPER64, FK_ZTRI64, FK_XINV64, FK_RES64,
    FK_TILE_FLAGS, FK_MOM_UMAX, FK_MOMENTUM, FK_RES_ENDS, FK_XRES_NORM32, FK_XINV_ACC32,
    FK_VOF_REC, FK_VOF_FLUX, FK_VOF_UPDATE, FK_COUNT
};

struct flups_plan_s {
    int nx, ny, nz, bc, prec, dev;
    int bcx, bcy;                // flups_xy_bc of the x and y ends (FLUPS_XY_PERIODIC unless created with ends)
    int Wx;                      // spectral columns along x: nx/2+1 (periodic x) or nx (Neumann/Dirichlet x)
    int xpack;                   // see Geo::xpack
    double dx, dy;
    cudaStream_t stream;
    int M, nxh, ldS;
    size_t npts, nspec;
    FftLen lx, ly, lz;           // lengths M (complex along x), ny, nz
    FftLen ly2;                  // ny/2 (mixed ends along y)
    // workspace
    void* spec;                  // spectrum, float2 or double2
    void* zscr;                  // z Thomas multipliers (walls)
    double* bx; double* by; double* bz;
    long long* trange;           // stencil tile density ranges (see FLUPS_TY)
    DevScalars* sc;              // device scalars
    DevScalars* sc_host;         // pinned host mirror
    double* part;                // reduction partials
    double* fin;                 // per-block sums of the final reduction (3 x 256)
    size_t npart;
    // tables (device)
    void* twx; void* twxr; void* twy; void* twz;   // W_M, W_nx (k<=M), W_ny, W_nz in compute type
    double* tabs64;              // [6][nz]: idzf, az, cz, idzc, dzf, dd = 2sx + 2sy + az + cz
    void* lamx; void* lamy; void* lamz;             // eigenvalues / norm, compute type
    void* twqx; void* twqy;      // ends in x, y: exp(-i pi k/(2n)) (k <= n/2 along x, k < ny along y), or for mixed
                                 // ends the pre-twiddles exp(-i pi (4m+1)/(4n)) then the post-twiddles exp(-i pi k/n)
    void* twy2;                  // W_{ny/2} twiddles (mixed ends along y)
    double* rbuf;                // FP64 defect of the FP32+refine solve with ends (npts)
    float* p32;                  // the first FP32 iterate in binary32 (npts), where p32_path holds
    long long* fq;               // F - MF of f at the first defect's scale (npts), where p32_path holds
    int fq_live;                 // fq written in the current solve; host-side state
    int p32_live;                // p32 holds the current iterate (p not yet written); host-side state
    void* tri;                   // walls: a_k/norm, b_k/norm, c_k/norm, compute type (3*nz)
    double sum_dzf;
    double dz0;                  // dzf[0] (the spacing of a periodic z)
    int uniform_h;               // dx == dy == every dzf: the exact fixed-point defect applies
    int density_set;
    // host-buffer (end-to-end) path, allocated on first use
    double* hbuf;                // 8 fields: u v w rho pn pnm1 f p
    double* hsol;                // host-buffer solve: 2 fields f p (allocated on first use)
    void* vofbuf;                // VoF step: cell records, face fluxes, three stages (first use)
    cudaStream_t cstream;        // copies that overlap the plan stream's kernels
    cudaEvent_t hev[3];          // call start, rho copied, every input copied (then: p ready)
    size_t total_bytes;
    void** allocs;               // every workspace allocation, freed by destroy
    int nallocs;
    unsigned long long launches; // kernels launched on this plan so far
    // TMA descriptors of the FP32 spectrum [nz][ny][ldS] for the pipelined column passes:
    // boxes of (B kx, up to 256 ky, 1 k) and (B kx, 1 ky, up to 256 k)
    CUtensorMap tm_y;            // (the type carries the 128-byte alignment TMA needs)
    CUtensorMap tm_z;
    int tma_ok;
    int* skip_ptr;               // passed to kernels as Geo::skip (set by the fixed-iteration solve)
    int cta_cap;                 // thread cap of the transform CTAs (autotuned per size in batches)
    int last_max_iter;           // max_iter of the last graph-capturable solve
    // exact variable-coefficient solve (flups_varcoef_solve), allocated on first use
    void* vcbuf;                 // face coefficients cx, cy, cz and PCG vectors r, z, d, q + scalars
    void* vcs_host;              // pinned host mirror of the PCG scalars
    // per-kernel timing
    int prof_on, prof_n, prof_cap, prof_open;
    cudaEvent_t* prof_ev;        // 2 * prof_cap events
    int* prof_kid;               // kernel id of each recorded pair
    double prof_ms[FK_COUNT];
    long long prof_cnt[FK_COUNT];
};

// Every launcher adds the number of kernels it launched to P->launches.
#define FLUPS_COUNT(P, n) ((P)->launches += (unsigned long long)(n))

void flups_prof_begin(flups_plan P, int kid);
void flups_prof_end(flups_plan P);

// Launchers (return cudaGetLastError()).
cudaError_t launch_set_density(flups_plan P, const double* rho, double rho0);
cudaError_t launch_rhs(flups_plan P, const double* u, const double* v, const double* w,
                       const double* pn, const double* pnm1, double c1, double c2, double dt, double* f);
cudaError_t launch_correct(flups_plan P, const double* p, const double* pn, const double* pnm1,
                           double c1, double c2, double dt, double* u, double* v, double* w);
// FP64 direct solve
cudaError_t launch_solve64(flups_plan P, const double* f, double* p);
// FP64 direct solve of a plan with Neumann or Dirichlet ends in x or y
cudaError_t launch_solve64_r2r(flups_plan P, const double* f, double* p);
// FP32+refine pieces of such plans: the FP64 defect (pass 1; pass 0: volume sum of f) with one
// partial sum per block in P->part, the FP32 solve of L d = r into p (or p += d), p += c.
int ends_res_blocks(flups_plan P);
cudaError_t launch_ends_residual(flups_plan P, const double* f, const double* p, double* r, double mf, int pass);
cudaError_t launch_ends_solve32(flups_plan P, const double* r, double* p, int acc);
cudaError_t launch_add_const(flups_plan P, double* a, double c);
// FP32 pipeline pieces
cudaError_t launch_xfwd32_from_f(flups_plan P, const double* f);            // S = FFTx(f), partial sums of f
cudaError_t launch_finalize_f(flups_plan P);                                 // mean_f, ||f - mean||^2
cudaError_t launch_xfwd32_residual(flups_plan P, const double* f, const double* p);  // S = FFTx(r), ||r||^2 partials
cudaError_t launch_xres_norm32(flups_plan P, const double* f, const double* p);     // ||r||^2 partials only
bool xres_norm_first(flups_plan P);     // later stopping tests take the norm-only pass first
cudaError_t launch_finalize_r(flups_plan P);
cudaError_t launch_yz_solve32(flups_plan P);                                 // y fwd, z solve, y inv on S
// 0: p = FFTx^-1(S) (+ mean); 1: p += . - mean; 2: p += .; 4: as 0, kept in binary32 in P->p32
// where the plan has one (mode 1 then reads it from there)
cudaError_t launch_xinv32(flups_plan P, double* p, int mode);
// p = P->p32 while the binary32 iterate is live (cond: only once the stopping test passed)
cudaError_t launch_p_from32(flups_plan P, double* p, bool cond);
// FP32+refine solve with a fixed sequence of kernels and no host synchronisation (graph
// capturable): after max_iter FP32 solves at most, the last defect norm is in P->sc.
cudaError_t launch_solve32_fixed(flups_plan P, const double* f, double* p, double rtol, int max_iter);
int flups_default_cta();
// FP64 residual (report only)
cudaError_t launch_residual64_norm(flups_plan P, const double* f, const double* p);

Geo plan_geo(flups_plan P);
// Remembers the last CUDA error the library observed (flups_last_cuda_error).
void flups_note_cuda_error(cudaError_t e);
// Tile width (log2) of the pipelined column passes for length N and M = nx/2 columns (kind 0:
// y transform, 1: periodic z solve).
int flups_pipe_lgB(int N, int M, int kind);
// Four-step FP32 column transforms (cols_kernels.cu): tile width (log2) for length N, or -1
// where the kernel does not apply; launch_cols4 runs the y transform (kind 0, inv picks the
// direction) or the periodic z solve (kind 1) on the plan's spectrum and returns false
// without launching where the kernel does not apply.
// One member of a batched ensemble solve (the stage kernels of fft_kernels.cu walk the
// concatenated (member, tile) lists of all members; 256 threads per CTA).  Filled on the host
// from the member's plan.
#define FLUPS_BATCH_THREADS 256
struct BatchMember {
    Geo g;                              // g.skip = &sc->done
    FftLen lx, ly, lz;                  // packed radix codes
    const float2 *twx, *twxr, *twy, *twz;
    const float *lamx, *lamy, *lamz, *tri;
    float2* spec;
    float* zscr;
    const double* f;
    double* p;
    DevScalars* sc;
    double* part;
    const double* dd;                   // diagonal of the z operator (FP64 defect)
    double nrm_w, npts;                 // 1 / (nx ny sum dzf), nx ny nz
    int ex, ey, ez;                     // elements per thread of the x, y, z transforms (8 or 12)
    int lgx, lgy, lgz;                  // log2 tile widths: 2^lg N / e = FLUPS_BATCH_THREADS
    int dmode;                          // defect: 2 (one spacing, fixed point) or 1 (FP64)
    int xr4;                            // forward x transform by the register four-step rows (M = 64)
    unsigned smx, smy, smz;             // dynamic shared memory of a tile of the x, y, z stages
    // the defect stage: z-marching fixed-point rows (zm = 1: G = zg groups of M threads, kz planes
    // per tile, zbx row blocks of 8 G rows per plane) or the untiled body (zm = 0, tiles as x)
    int zm, zg, zkz, zbx, td;
    unsigned smd;
    int tx, ty, tz;                     // tiles of the x, y, z stages
    int ymain, zmain, xq;               // main tiles of the y and z stages; x tiles per plane row set
};
// Batched stages (fft_kernels.cu).  o*: the work list of the x, y, z and defect stages (device
// memory), item b = (member << 20) | tile, members in order; smem_*: the largest dynamic shared
// memory a member's tile of that stage needs.
struct BatchLaunch {
    const BatchMember* mem;
    const unsigned *ox, *oy, *oz, *od;
    int n, total_x, total_y, total_z, total_d;
    size_t smem_x, smem_y, smem_z, smem_d;
    cudaStream_t stream;
};
// The fixed FP32 + FP64-defect sequence of every member (as launch_solve32_fixed) with one
// kernel per stage; returns the kernels launched, or -1 on a launch error.
int launch_batch_fixed(const BatchLaunch& L, double rtol, int max_iter);
// The same sequence captured as a graph in which every iteration after the first sits in a
// conditional (IF) node that runs only while some member has not converged (aux: a second
// stream for the nodes' bodies).  Returns the kernels in the graph, or -1 (nothing captured).
int capture_batch_graph(const BatchLaunch& L, cudaStream_t aux, double rtol, int max_iter, cudaGraph_t* out);
// Whether a plan's member can take the batched stages (x, y periodic; lengths 8 * 2^a or 12 * 2^a;
// FP32 + refine).
bool batch_member_ok(flups_plan P);
void batch_member_fill(flups_plan P, const double* f, double* p, BatchMember* out);

// Register four-step x-row kernels (xrow_kernels.cu) for M = nx / 2 in {64, ..., 1024}: rows
// per CTA (0: not available); forward from f (stats: the partial sums of the first pass) and
// inverse (mode 0: p = x with the mean's partial sums, 1: p += x - <p_0>, 2: p += x, 3: p = x;
// 4: as 0 with x stored in binary32 to P->p32, 5: as 1 with the old iterate read from P->p32).
int xrow4_rows(int M);
// Whether the FP32+refine solve keeps its first iterate in binary32 (P->p32): one-spacing grids
// whose first defect takes the z-marching kernel and whose inverse x takes the register rows.
bool p32_path(int M, int ny);
bool launch_xrow4_fwd(flups_plan P, const double* f, const Geo& g, bool stats);
bool launch_xrow4_inv(flups_plan P, double* p, const Geo& g, int mode);
int cols4_lgB(int N, int M, int kind);
bool launch_cols4(flups_plan P, float2* S, const Geo& g, int kind, bool inv);
// Walls z solve in FP32 without HBM scratch (cols_kernels.cu): tile width (log2) of its TMA
// boxes for nz rows, or -1 where it does not apply; launch_ztri_tile returns the number of
// kernels it launched (0: not applicable, nothing launched).
int ztri_tile_lgB(int nz);
int launch_ztri_tile(flups_plan P, float2* S, const Geo& g);
