// C ABI and host orchestration of the MRCM-OS library (include/mrcm.h).
//
// The host side plans the decomposition (subdomain boxes, oversampled boxes,
// colours, interface numbering and slabs), owns every device allocation of a
// handle, and issues the kernels on the caller's stream.  All arithmetic of
// the method runs in the CUDA kernels of this library.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "../../include/mrcm.h"
#include "mrcm_internal.cuh"

// launchers defined in the other translation units
size_t local2d_smem(int prec, int nx, int ny, int nrhs, bool part);
size_t smooth2d_smem(int prec, int nx, int ny);
size_t spack_bytes(int prec, int nx, int ny);
int local2d_class(int prec, int nx);
cudaError_t launch_local2d(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs, int bw,
                           size_t smem, cudaStream_t s);
cudaError_t launch_smooth2d(const DevPtrs& P, const MethodDev& M, const int* items, int nitems,
                            size_t smem, cudaStream_t s);
cudaError_t launch_assemble2d(const DevPtrs& P, const double* X, int nitems, int ncell_i_max,
                              cudaStream_t s);
cudaError_t launch_faces(const MemberDev* dmem, int nmem, long long maxcells, const double* K, double* Tf,
                         double* hk, double* wh, cudaStream_t s);
cudaError_t launch_output(const MemberDev* dmem, int nmem, int member, const double* p, const double* u,
                          long long off, long long nc, int nside, double* dmean, double* pout,
                          double* uout, cudaStream_t s);

cudaError_t if_assemble(const DevPtrs& P, const MethodDev& M, const IfPtrs& I, int nitems, int nrows,
                        cudaStream_t s);
cudaError_t bcr_fill(const IfPtrs& I, int nslab, cudaStream_t s);
cudaError_t bcr_elim(const IfPtrs& I, const ElimDev* el, int nel, size_t smem, cudaStream_t s);
cudaError_t if_residual(const IfPtrs& I, const int* row_member, int nrows, int first, cudaStream_t s);
cudaError_t bcr_fwd(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s);
cudaError_t bcr_bwd(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s);
cudaError_t if_update(const IfPtrs& I, int ncols, cudaStream_t s);
cudaError_t kry_to_bq(const IfPtrs& I, const double* v, int n, cudaStream_t s);
cudaError_t kry_from_bq(const IfPtrs& I, double* z, int n, cudaStream_t s);
cudaError_t kry_axpby(double* y, const double* x, double a, double b, int n, cudaStream_t s);
cudaError_t kry_dot(const double* a, const double* b, int n, double* part, cudaStream_t s);
int kry_blocks();
cudaError_t kry_mdot(const double* V, const double* w, int n, int nv, double* part, cudaStream_t s);
cudaError_t kry_msub(double* w, const double* V, const double* coef, int nv, int n, cudaStream_t s);
cudaError_t lu_inverse(const IfPtrs& I, const ElimDev* el, int nel, int* status, int variant, cudaStream_t s);
int slab_inverse_gj_ok(int npad);
int slab_inverse_gjr_npad(int npad);
size_t elim_smem_bytes(int nmv, int cw);
size_t lu_smem(int np, int xch);
size_t local3d_smem(int prec, int nx, int ny, int nz, bool part);
size_t smooth3d_smem(int prec, int nx, int ny, int nz);
size_t factor3_entries(int nx, int ny, int nz);
bool stage3_aligned(int prec, int nx, int ny, int nz);
cudaError_t launch_local3d(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs, size_t smem,
                           cudaStream_t s);
cudaError_t launch_smooth3d(const DevPtrs& P, const MethodDev& M, const int* items, int nitems, size_t smem,
                            cudaStream_t s);
cudaError_t launch_assemble3d(const DevPtrs& P, const double* X, int nitems, int ncell_i_max, cudaStream_t s);
cudaError_t if_residualT(const IfPtrs& I, const SubDev* sub, const int* col_item, const double* z,
                         const double* y, const int* row_member, int n, int first, cudaStream_t s);
cudaError_t bcr_bwdT(const IfPtrs& I, const ElimDev* el, int nel, int nmax, int up, cudaStream_t s);
cudaError_t bcr_fwdT(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s);
cudaError_t if_updateT(const IfPtrs& I, double* y, int n, cudaStream_t s);
size_t adj_smooth2d_smem(int prec, int nx, int ny);
size_t adj_local2d_smem(int prec, int nx, int ny, int nw, bool part);
cudaError_t launch_adj_smooth2d(const DevPtrs& P, const MethodDev& M, const AdjPtrs& A, const int* items,
                                int nitems, size_t smem, cudaStream_t s);
cudaError_t launch_adj_assemble2d(const DevPtrs& P, const AdjPtrs& A, int nitems, int ncell_i_max,
                                  cudaStream_t s);
cudaError_t launch_adj_moments(const DevPtrs& P, const MethodDev& M, const AdjPtrs& A, int nitems,
                               cudaStream_t s);
cudaError_t launch_adj_local2d(const DevPtrs& P, const MethodDev& M, const AdjPtrs& A, const Job* jobs,
                               int njobs, int bw, int nw, size_t smem, cudaStream_t s);
cudaError_t launch_grad_logK(const MemberDev* dmem, int nmem, long long maxcells, const double* K,
                             const double* Tf, const double* hk, const AdjPtrs& A, double* out, cudaStream_t s);
cudaError_t launch_set_K(const double* src, double* K, long long n, int is_log, int* status, cudaStream_t s);

namespace {

enum Stage { ST_CREATED = 0, ST_BASIS = 1, ST_SOLVED = 2 };

struct JobClass {
    int bw;
    size_t smem;
    int off, count;
};

struct Level {
    int off, count;           // into the elimination array
};

struct AdjClass {
    int bw, nw;
    size_t smem;
    int off, count;
};

// Workspace of the reverse pass, allocated by the first mrcm_adjoint call.
struct AdjWork {
    bool ready = false;
    AdjPtrs A{};
    int* col_item = nullptr;
    Job* jobs = nullptr;
    std::vector<AdjClass> classes;
    size_t smooth_smem = 0;
    double* snap = nullptr;
    size_t snap_len = 0;      // doubles
    double* gout = nullptr;   // device result when the caller passes host memory
};

}  // namespace

struct mrcm_handle {
    cudaStream_t stream = 0;
    int device = 0;               // the device current at creation (all of the handle's memory lives there)
    mrcm_params prm{};
    int dim = 2;
    int count = 0;
    std::string err;
    int stage = ST_CREATED;
    // plan
    std::vector<MemberDev> mem;
    std::vector<SubDev> sub;
    std::vector<SlabDev> slabs;
    std::vector<ElimDev> elims;
    std::vector<Level> levels;   // last level = roots
    std::vector<JobClass> jclasses;
    std::vector<int> colour_off; // colour c items: [colour_off[c], colour_off[c+1])
    size_t smooth_smem = 0;
    int nbasis_max = 0, ncell_i_max = 0, side_max = 0, npsi = 1;
    long long ncells = 0;
    int nif = 0, npad = 0, nmax_slab = 0;
    size_t elim_smem = 0;
    MethodDev mth{};
    // device
    MemberDev* d_mem = nullptr;
    SubDev* d_sub = nullptr;
    Job* d_jobs = nullptr;
    int* d_colour_items = nullptr;
    double *d_K = nullptr, *d_f = nullptr, *d_p = nullptr, *d_u = nullptr;
    double *d_Tf = nullptr, *d_hk = nullptr, *d_wh = nullptr;
    void* d_fac = nullptr;
    void* d_fac_aux = nullptr;
    void* d_fac_part = nullptr;
    double* d_dsc = nullptr;
    double *d_Psi = nullptr, *d_Ug = nullptr, *d_pbar = nullptr, *d_ubg = nullptr, *d_mom = nullptr;
    int* d_status = nullptr;
    double* d_mean = nullptr;
    DevPtrs P{};
    // interface
    IfPtrs I{};
    SlabDev* d_slabs = nullptr;
    ElimDev* d_elims = nullptr;
    int* d_row_member = nullptr;
    std::vector<void*> allocs;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_rec;
    long long launches[7] = {0, 0, 0, 0, 0, 0, 0};
    // captured step
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr, user_stream = nullptr;
    // the basis build's job classes run concurrently: one stream per class
    // beyond the first, forked from and joined to the handle's stream
    std::vector<cudaStream_t> class_streams;
    std::vector<cudaEvent_t> class_events;   // [0] fork, [1 + k] join of class stream k
    int graph_steps = -1, graph_nit = 0;
    // reverse pass
    AdjWork adj;
    int smooth_steps = 0;     // smoothing steps applied since the last interface solve
    // stats
    int if_iters = 0;
    double if_res = 0.0;
    bool if_krylov = false;       // the last interface solve needed the GMRES fallback
    int slab_variant = -1;        // slab inverses: -1 not chosen yet, 0 blocked Gauss-Jordan, 1 LU,
                                  // 2 register-resident Gauss-Jordan (autotuner)
    int tune_source = 0;          // 0 none, 1 from the tuning cache, 2 measured by this handle
    double tune_ms[3] = {0.0, 0.0, 0.0};   // measured device ms (factor + refine) of each variant
    double* d_kry = nullptr;      // its workspace (allocated on first use)
    int loc_ir = 0;
    long long local_solves = 0;
    int call_depth = 0;           // nesting of public calls (the metrics line is written by the outermost)
};

namespace {

int fail(mrcm_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

#define CUDA_TRY(h, call)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail((h), MRCM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

cudaEvent_t take_event(mrcm_handle* h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

// Records device time of one phase when profiling is on.
struct Phase {
    mrcm_handle* h;
    int ph;
    cudaEvent_t a = nullptr;
    Phase(mrcm_handle* hh, int p) : h(hh), ph(p) {
        if (h->prof) {
            a = take_event(h);
            if (a) cudaEventRecord(a, h->stream);
        }
    }
    ~Phase() {
        if (h->prof && a) {
            cudaEvent_t b = take_event(h);
            if (b) {
                cudaEventRecord(b, h->stream);
                h->ev_rec.push_back({ph, {a, b}});
            }
        }
    }
};

template <typename T>
int dalloc(mrcm_handle* h, T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * count);
    if (e != cudaSuccess) return fail(h, MRCM_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->allocs.push_back(q);
    *p = (T*)q;
    return 0;
}

int check_inputs(mrcm_handle* h, const mrcm_grid* g, const mrcm_bc* bc, const mrcm_partition* pt,
                 const mrcm_params* pr) {
    if (!g || !bc || !pt || !pr) return fail(h, MRCM_ERR_BAD_INPUT, "null argument");
    if (g->dim != 2 && g->dim != 3) return fail(h, MRCM_ERR_BAD_INPUT, "dim must be 2 or 3");
    for (int a = 0; a < g->dim; ++a) {
        if (g->n[a] <= 0 || !(g->h[a] > 0.0) || !std::isfinite(g->h[a]))
            return fail(h, MRCM_ERR_BAD_INPUT, "grid sizes must be positive");
        if (pt->sub[a] <= 0 || g->n[a] % pt->sub[a])
            return fail(h, MRCM_ERR_BAD_INPUT, "subdomain size must divide the grid");
        if (pt->overlap < 0 || 2 * pt->overlap >= pt->sub[a])
            return fail(h, MRCM_ERR_BAD_INPUT, "need 0 <= 2*overlap < subdomain size");
    }
    for (int s = 0; s < 2 * g->dim; ++s)
        if (bc->kind[s] != MRCM_NEUMANN && bc->kind[s] != MRCM_DIRICHLET)
            return fail(h, MRCM_ERR_BAD_INPUT, "bad boundary kind");
    if (pr->space != MRCM_P0 && pr->space != MRCM_P1) return fail(h, MRCM_ERR_BAD_INPUT, "bad space");
    if (pr->precision != MRCM_FP64 && pr->precision != MRCM_MIXED)
        return fail(h, MRCM_ERR_BAD_INPUT, "bad precision");
    if (!(pr->alpha_basis > 0.0) || !(pr->alpha_smooth > 0.0))
        return fail(h, MRCM_ERR_BAD_INPUT, "alpha must be positive");
    if (pr->max_ir < 1) return fail(h, MRCM_ERR_BAD_INPUT, "max_ir must be >= 1");
    if (pr->particular != MRCM_PARTICULAR_OMEGA && pr->particular != MRCM_PARTICULAR_HAT)
        return fail(h, MRCM_ERR_BAD_INPUT, "bad particular");
    return 0;
}

// -------------------------------------------------------------------------
// planning
// -------------------------------------------------------------------------
int plan(mrcm_handle* h, const mrcm_grid* grids, const mrcm_bc* bcs, const mrcm_partition* parts) {
    const int d = h->dim;
    const int npsi = h->prm.space == MRCM_P0 ? 1 : (d == 2 ? 2 : 3);
    h->npsi = npsi;
    long long cell_off = 0;
    int if_off = 0;
    for (int m = 0; m < h->count; ++m) {
        const mrcm_grid& g = grids[m];
        const mrcm_bc& bc = bcs[m];
        const mrcm_partition& pt = parts[m];
        MemberDev md{};
        md.dim = d;
        long long nc = 1;
        for (int a = 0; a < 3; ++a) {
            md.n[a] = a < d ? g.n[a] : 1;
            md.h[a] = a < d ? g.h[a] : 1.0;
            md.sub[a] = a < d ? pt.sub[a] : 1;
            md.M[a] = md.n[a] / md.sub[a];
            md.Hw[a] = md.sub[a] * md.h[a];
            nc *= md.n[a];
        }
        md.overlap = pt.overlap;
        md.pure_neumann = 1;
        for (int s = 0; s < 6; ++s) {
            md.bc_kind[s] = s < 2 * d ? bc.kind[s] : MRCM_NEUMANN;
            md.bc_val[s] = s < 2 * d ? bc.value[s] : 0.0;
            if (s < 2 * d && bc.kind[s] == MRCM_DIRICHLET) md.pure_neumann = 0;
        }
        md.cell_off = cell_off;
        md.sub0 = (int)h->sub.size();
        md.nsub = md.M[0] * md.M[1] * md.M[2];
        md.if0 = if_off;
        if (md.nsub < 2) return fail(h, MRCM_ERR_BAD_INPUT, "need at least two subdomains");
        for (int idx = 0; idx < md.nsub; ++idx) {
            SubDev sd{};
            sd.member = m;
            int r = idx;
            for (int a = 0; a < 3; ++a) {
                sd.multi[a] = r % md.M[a];
                r /= md.M[a];
            }
            sd.side_mask = 0;
            sd.colour = 0;
            for (int a = 0; a < 3; ++a) {
                sd.lo[a] = sd.multi[a] * md.sub[a];
                sd.hi[a] = sd.lo[a] + md.sub[a];
                sd.loh[a] = a < d ? std::max(0, sd.lo[a] - pt.overlap) : 0;
                sd.hih[a] = a < d ? std::min(md.n[a], sd.hi[a] + pt.overlap) : 1;
                if (a < d) {
                    if (sd.multi[a] > 0) sd.side_mask |= 1 << (2 * a);
                    if (sd.multi[a] < md.M[a] - 1) sd.side_mask |= 1 << (2 * a + 1);
                    sd.colour |= (sd.multi[a] & 1) << a;
                }
            }
            int nsides = __builtin_popcount(sd.side_mask);
            sd.nbasis = nsides * npsi;
            sd.col0 = if_off;
            if_off += sd.nbasis;
            for (int s = 0; s < 6; ++s) {
                sd.nbr[s] = -1;
                if (sd.side_mask & (1 << s)) {
                    int a = s >> 1;
                    int stride = 1;
                    for (int b = 0; b < a; ++b) stride *= md.M[b];
                    sd.nbr[s] = md.sub0 + idx + ((s & 1) ? stride : -stride);
                }
            }
            h->sub.push_back(sd);
            h->nbasis_max = std::max(h->nbasis_max, sd.nbasis);
            int nci = 1;
            for (int a = 0; a < d; ++a) nci *= md.sub[a];
            h->ncell_i_max = std::max(h->ncell_i_max, nci);
            for (int a = 0; a < d; ++a) {
                int face = 1;
                for (int b = 0; b < d; ++b)
                    if (b != a) face *= md.sub[b];
                h->side_max = std::max(h->side_max, face);
            }
        }
        md.nif = if_off - md.if0;
        // interface slabs along the last axis
        const int la = d - 1;
        const int S = md.M[la];
        const int per = md.nsub / S;
        md.slab0 = (int)h->slabs.size();
        md.nslab = S;
        int ldc = 0;
        for (int j = 0; j < S; ++j) {
            SlabDev sl{};
            sl.member = m;
            sl.col0 = h->sub[md.sub0 + j * per].col0;
            int n = 0;
            for (int q = 0; q < per; ++q) n += h->sub[md.sub0 + j * per + q].nbasis;
            sl.n = n;
            sl.up = j + 1 < S ? md.slab0 + j + 1 : -1;
            sl.dn = j > 0 ? md.slab0 + j - 1 : -1;
            ldc = std::max(ldc, n);
            h->slabs.push_back(sl);
        }
        for (int j = 0; j < S; ++j) h->slabs[md.slab0 + j].ldc = ldc;
        h->mem.push_back(md);
        cell_off += nc;
    }
    h->ncells = cell_off;
    h->nif = if_off;
    return 0;
}

// row (kind, side) of local row q of a subdomain, mirroring k_if_assemble
void row_kind(const SubDev& sd, int d, int npsi, int q, int* kind, int* sid) {
    *kind = -1;
    for (int a = 0; a < d; ++a) {
        int sh = 2 * a + 1;
        if (sd.side_mask & (1 << sh)) {
            if (q < npsi) { *kind = 0; *sid = sh; return; }
            q -= npsi;
        }
    }
    for (int a = 0; a < d; ++a) {
        int sl = 2 * a;
        if (sd.side_mask & (1 << sl)) {
            if (q < npsi) { *kind = 1; *sid = sl; return; }
            q -= npsi;
        }
    }
}

}  // namespace

// -------------------------------------------------------------------------
// creation
// -------------------------------------------------------------------------
static int create_impl(int count, const mrcm_grid* grids, const double* const* K, const double* const* f,
                       const mrcm_bc* bcs, const mrcm_partition* parts, const mrcm_params* params,
                       int device_ptrs, void* stream, mrcm_handle** out) {
    if (!out) return MRCM_ERR_BAD_INPUT;
    *out = nullptr;
    mrcm_handle* h = new mrcm_handle();
    *out = h;
    if (count < 1 || !grids || !K || !f || !bcs || !parts || !params)
        return fail(h, MRCM_ERR_BAD_INPUT, "bad arguments");
    h->stream = (cudaStream_t)stream;
    h->user_stream = h->stream;
    h->prm = *params;
    h->count = count;
    h->dim = grids[0].dim;
    for (int m = 0; m < count; ++m) {
        int rc = check_inputs(h, &grids[m], &bcs[m], &parts[m], params);
        if (rc) return rc;
        if (grids[m].dim != h->dim) return fail(h, MRCM_ERR_BAD_INPUT, "members must share dim");
    }
    int rc = plan(h, grids, bcs, parts);
    if (rc) return rc;
    for (int m = 0; m < count; ++m) {
        const MemberDev& md = h->mem[m];
        long long nc = (long long)md.n[0] * md.n[1] * md.n[2];
        if (!K[m] || !f[m]) return fail(h, MRCM_ERR_BAD_INPUT, "null K or f");
        if (!device_ptrs) {
            for (long long c = 0; c < nc; ++c)
                if (!(K[m][c] > 0.0) || !std::isfinite(K[m][c]) || !std::isfinite(f[m][c]))
                    return fail(h, MRCM_ERR_BAD_INPUT, "K must be positive and finite, f finite");
        }
    }
    const int d = h->dim;
    const int prec = h->prm.precision;
    const size_t tsz = prec == MRCM_FP64 ? sizeof(double) : sizeof(float);
    h->mth.space = h->prm.space;
    h->mth.npsi = h->npsi;
    h->mth.prec = prec;
    h->mth.alpha_b = h->prm.alpha_basis;
    h->mth.alpha_s = h->prm.alpha_smooth;
    h->mth.ir_tol = h->prm.ir_tol > 0 ? h->prm.ir_tol : 1e-12;
    h->mth.max_ir = prec == MRCM_FP64 ? 1 : h->prm.max_ir;
    h->mth.same_alpha = h->prm.alpha_basis == h->prm.alpha_smooth;
    h->mth.part_hat = h->prm.particular == MRCM_PARTICULAR_HAT;
    // The smoothing kernel waits up to 2^31 cycles for its staged copy.  For
    // the failure-detection test only, MRCM_TEST_FIRST_WAIT_CYCLES = N > 0
    // makes its first wait one of N cycles for a barrier nothing arrives at:
    // it runs out, the kernel waits again at the full limit for the copy in
    // flight, skips its solve and flags it (MRCM_ERR_TIMEOUT).
    h->mth.wait0 = 0;
    if (const char* w = std::getenv("MRCM_TEST_FIRST_WAIT_CYCLES"))
        if (*w) h->mth.wait0 = std::max(0LL, std::atoll(w));

    // jobs: basis, particular, smoothing factor
    std::map<int, std::vector<Job>> byw;
    std::map<int, size_t> smem_w;
    size_t fac_stride = 0, dsc_stride = 0, part_stride = 0;
    const int nitems = (int)h->sub.size();
    for (int s = 0; s < nitems; ++s) {
        const SubDev& sd = h->sub[s];
        int bx = sd.hih[0] - sd.loh[0], by = sd.hih[1] - sd.loh[1], bz = sd.hih[2] - sd.loh[2];
        int ix = sd.hi[0] - sd.lo[0], iy = sd.hi[1] - sd.lo[1], iz = sd.hi[2] - sd.lo[2];
        if (d == 3) {
            // one class; boxes are factored plane by plane with the factor in global memory
            const int pb = bx * by * bz / std::max({bx, by, bz});
            if (pb > 256) return fail(h, MRCM_ERR_UNSUPPORTED, "3D boxes with planes of more than 256 cells");
            if (!stage3_aligned(prec, bx, by, bz) || !stage3_aligned(prec, ix, iy, iz))
                return fail(h, MRCM_ERR_UNSUPPORTED, "3D box layout breaks the 16-byte rule of the bulk copies");
            fac_stride = std::max(fac_stride, (factor3_entries(bx, by, bz) + 3) & ~size_t(3));
            dsc_stride = std::max(dsc_stride, (size_t)bx * by * bz);
            byw[0].push_back(Job{s, JOB_BASIS});
            smem_w[0] = std::max(smem_w[0], local3d_smem(prec, bx, by, bz, false));
            if (!h->mth.part_hat) {
                // the particular problem on Omega_i, with its own factor (on
                // hat-Omega_i it is the basis job's last right-hand side)
                part_stride = std::max(part_stride, (factor3_entries(ix, iy, iz) + 3) & ~size_t(3));
                byw[0].push_back(Job{s, JOB_PART});
                smem_w[0] = std::max(smem_w[0], local3d_smem(prec, ix, iy, iz, true));
            }
            if (!h->mth.same_alpha) byw[0].push_back(Job{s, JOB_SFACT});
            h->smooth_smem = std::max(h->smooth_smem, smooth3d_smem(prec, bx, by, bz));
            continue;
        }
        if (bx > 32 || ix > 32)
            return fail(h, MRCM_ERR_UNSUPPORTED, "2D boxes wider than 32 cells along x are not supported");
        fac_stride = std::max(fac_stride, spack_bytes(prec, bx, by) / tsz);   // smoothing packs, 16-byte multiples
        dsc_stride = std::max(dsc_stride, (size_t)bx * by);
        // with the particular problem on hat-Omega_i it is one more
        // right-hand side of the basis job (kept in global memory, so the
        // basis box needs no more shared memory)
        const bool hat = h->mth.part_hat;
        auto add = [&](int type, int nx, int ny, int nrhs, bool staged) {
            const int bw = local2d_class(prec, nx);
            byw[bw].push_back(Job{s, type});
            smem_w[bw] = std::max(smem_w[bw], local2d_smem(prec, nx, ny, std::max(std::min(nrhs, 4), 1), staged));
        };
        add(JOB_BASIS, bx, by, sd.nbasis + (hat ? 1 : 0), false);
        if (!hat) add(JOB_PART, ix, iy, 1, true);
        if (!h->mth.same_alpha) add(JOB_SFACT, bx, by, 0, false);
        h->smooth_smem = std::max(h->smooth_smem, smooth2d_smem(prec, bx, by));
    }
    if (h->smooth_smem > 227 * 1024) return fail(h, MRCM_ERR_UNSUPPORTED, "subdomain box too large for shared memory");
    std::vector<Job> jobs;
    for (auto& kv : byw) {
        JobClass jc{kv.first, smem_w[kv.first], (int)jobs.size(), (int)kv.second.size()};
        if (jc.smem > 227 * 1024) return fail(h, MRCM_ERR_UNSUPPORTED, "subdomain box too large for shared memory");
        h->jclasses.push_back(jc);
        jobs.insert(jobs.end(), kv.second.begin(), kv.second.end());
    }
    // colours
    std::vector<int> citems;
    h->colour_off.assign((1 << d) + 1, 0);
    for (int c = 0; c < (1 << d); ++c) {
        h->colour_off[c] = (int)citems.size();
        for (int s = 0; s < nitems; ++s)
            if (h->sub[s].colour == c) citems.push_back(s);
    }
    h->colour_off[1 << d] = (int)citems.size();

    // ---- device allocations ----
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(h, MRCM_ERR_CUDA, "no current CUDA device");
    int e = 0;
    const int nmem = (int)h->mem.size();
    if ((e = dalloc(h, &h->d_mem, nmem))) return e;
    if ((e = dalloc(h, &h->d_sub, nitems))) return e;
    if ((e = dalloc(h, &h->d_jobs, jobs.size()))) return e;
    if ((e = dalloc(h, &h->d_colour_items, citems.size()))) return e;
    if ((e = dalloc(h, &h->d_K, h->ncells))) return e;
    if ((e = dalloc(h, &h->d_f, h->ncells))) return e;
    if ((e = dalloc(h, &h->d_p, h->ncells))) return e;
    if ((e = dalloc(h, &h->d_u, h->ncells * 2 * d))) return e;
    if ((e = dalloc(h, &h->d_Tf, h->ncells * 3))) return e;
    if ((e = dalloc(h, &h->d_hk, h->ncells * 3))) return e;
    if ((e = dalloc(h, &h->d_wh, h->ncells * 3))) return e;
    if ((e = dalloc(h, (char**)&h->d_fac, fac_stride * nitems * tsz))) return e;
    double* d_xs = nullptr;
    if (d == 3) {
        if ((e = dalloc(h, (char**)&h->d_fac_part, part_stride * nitems * tsz))) return e;
        if (!h->mth.same_alpha && (e = dalloc(h, (char**)&h->d_fac_aux, fac_stride * nitems * tsz))) return e;
        // FP64 iterates of the local solves: one slot of 4 right-hand sides per CTA of the largest launch
        const size_t slots = std::max(jobs.size(), (size_t)nitems);
        if ((e = dalloc(h, &d_xs, slots * 4 * dsc_stride))) return e;
    }
    if ((e = dalloc(h, &h->d_dsc, dsc_stride * nitems))) return e;
    double* d_bsrc = nullptr;
    if (h->mth.part_hat && (e = dalloc(h, &d_bsrc, dsc_stride * nitems))) return e;
    if ((e = dalloc(h, &h->d_Psi, (size_t)nitems * h->nbasis_max * h->ncell_i_max))) return e;
    if ((e = dalloc(h, &h->d_Ug, (size_t)nitems * h->nbasis_max * MRCM_MAXSIDE * h->side_max))) return e;
    if ((e = dalloc(h, &h->d_pbar, (size_t)nitems * h->ncell_i_max))) return e;
    if ((e = dalloc(h, &h->d_ubg, (size_t)nitems * MRCM_MAXSIDE * h->side_max))) return e;
    if ((e = dalloc(h, &h->d_mom, (size_t)nitems * (h->nbasis_max + 1) * MRCM_MAXSIDE * h->npsi * 2))) return e;
    if ((e = dalloc(h, &h->d_status, MRCM_STATUS_WORDS))) return e;
    if ((e = dalloc(h, &h->d_mean, nmem))) return e;
    cudaStream_t st = h->stream;
    CUDA_TRY(h, cudaMemcpyAsync(h->d_mem, h->mem.data(), sizeof(MemberDev) * nmem, cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_sub, h->sub.data(), sizeof(SubDev) * nitems, cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_jobs, jobs.data(), sizeof(Job) * jobs.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_colour_items, citems.data(), sizeof(int) * citems.size(),
                                cudaMemcpyHostToDevice, st));
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int m = 0; m < count; ++m) {
        const MemberDev& md = h->mem[m];
        long long nc = (long long)md.n[0] * md.n[1] * md.n[2];
        CUDA_TRY(h, cudaMemcpyAsync(h->d_K + md.cell_off, K[m], sizeof(double) * nc, kind, st));
        CUDA_TRY(h, cudaMemcpyAsync(h->d_f + md.cell_off, f[m], sizeof(double) * nc, kind, st));
    }
    {
        long long maxc = 0;
        for (auto& md : h->mem) maxc = std::max(maxc, (long long)md.n[0] * md.n[1] * md.n[2]);
        CUDA_TRY(h, launch_faces(h->d_mem, nmem, maxc, h->d_K, h->d_Tf, h->d_hk, h->d_wh, st));
    }
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * MRCM_STATUS_WORDS, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_p, 0, sizeof(double) * h->ncells, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_u, 0, sizeof(double) * h->ncells * 2 * d, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_mom, 0,
                                sizeof(double) * nitems * (h->nbasis_max + 1) * MRCM_MAXSIDE * h->npsi * 2, st));

    DevPtrs& P = h->P;
    P.mem = h->d_mem;
    P.sub = h->d_sub;
    P.K = h->d_K;
    P.f = h->d_f;
    P.Tf = h->d_Tf;
    P.hk = h->d_hk;
    P.wh = h->d_wh;
    P.p = h->d_p;
    P.u = h->d_u;
    P.fac = h->d_fac;
    P.fac_stride = (long long)fac_stride;
    P.fac_aux = h->d_fac_aux;
    P.fac_part = h->d_fac_part;
    P.part_stride = (long long)part_stride;
    P.xs = d_xs;
    P.xs_stride = (long long)(4 * dsc_stride);
    P.dsc = h->d_dsc;
    P.dsc_stride = (long long)dsc_stride;
    P.bsrc = d_bsrc;
    P.Psi = h->d_Psi;
    P.Ug = h->d_Ug;
    P.pbar = h->d_pbar;
    P.ubg = h->d_ubg;
    P.mom = h->d_mom;
    P.nbasis_max = h->nbasis_max;
    P.ncell_i_max = h->ncell_i_max;
    P.side_max = h->side_max;
    P.npsi = h->npsi;
    P.status = h->d_status;

    // ---- interface plan: slabs, row index lists, elimination levels ----
    std::vector<int> idxpool;
    long long offD = 0, offC = 0, offR = 0;
    int npad = 0;
    for (auto& sl : h->slabs) npad = std::max(npad, sl.n);
    npad = (npad + 3) & ~3;
    h->npad = npad;
    h->nmax_slab = npad;
    std::vector<int> row_member(h->nif);
    for (auto& md : h->mem)
        for (int r = md.if0; r < md.if0 + md.nif; ++r) row_member[r] = (int)(&md - &h->mem[0]);
    for (size_t j = 0; j < h->slabs.size(); ++j) {
        SlabDev& sl = h->slabs[j];
        const MemberDev& md = h->mem[sl.member];
        const int la = d - 1;
        std::vector<int> mrows, vrows, mpos(sl.n, -1), vpos(sl.n, -1);
        for (int s = md.sub0; s < md.sub0 + md.nsub; ++s) {
            const SubDev& sd = h->sub[s];
            if (sd.col0 < sl.col0 || sd.col0 >= sl.col0 + sl.n) continue;
            for (int q = 0; q < sd.nbasis; ++q) {
                int kind, sid;
                row_kind(sd, d, h->npsi, q, &kind, &sid);
                int rr = sd.col0 + q - sl.col0;
                if (kind == 0 && sid == 2 * la + 1) { mpos[rr] = (int)mrows.size(); mrows.push_back(rr); }
                if (kind == 1 && sid == 2 * la) { vpos[rr] = (int)vrows.size(); vrows.push_back(rr); }
            }
        }
        sl.nm = (int)mrows.size();
        sl.nv = (int)vrows.size();
        sl.offIdx = (long long)idxpool.size();
        idxpool.insert(idxpool.end(), mrows.begin(), mrows.end());
        idxpool.insert(idxpool.end(), vrows.begin(), vrows.end());
        idxpool.insert(idxpool.end(), mpos.begin(), mpos.end());
        idxpool.insert(idxpool.end(), vpos.begin(), vpos.end());
        sl.offD = offD;
        offD += (long long)npad * npad;
        sl.offCup = offC;
        sl.offCdn = offC + (long long)sl.nm * sl.ldc;
        offC += (long long)(sl.nm + sl.nv) * sl.ldc;
        sl.offRup = offR;
        sl.offRdn = offR + (long long)sl.ldc * sl.n;
        offR += 2LL * sl.ldc * sl.n;
        sl.offPiv = (long long)j * npad;
    }
    // Schur-update scratch: bounded by the largest couplings; the coupling
    // columns are staged in chunks that fit shared memory
    int elim_cw = npad, xch = 64;
    {
        size_t nmv = 0;
        for (auto& sl : h->slabs) nmv = std::max(nmv, (size_t)std::max(sl.nm, sl.nv));
        while (elim_cw > 32 && elim_smem_bytes((int)nmv, elim_cw) > 227 * 1024) elim_cw = (elim_cw + 1) / 2;
        h->elim_smem = elim_smem_bytes((int)nmv, elim_cw);
        if (h->elim_smem > 227 * 1024) return fail(h, MRCM_ERR_UNSUPPORTED, "interface coupling blocks too large");
        // 1 KB of the 227 KB per block is left to the slab LU's static shared memory
        while (xch > 4 && lu_smem(npad, xch) > 226 * 1024) xch /= 2;
        if (lu_smem(npad, xch) > 226 * 1024) return fail(h, MRCM_ERR_UNSUPPORTED, "interface slabs too large");
    }
    // elimination levels over all members
    int maxS = 0;
    for (auto& md : h->mem) maxS = std::max(maxS, md.nslab);
    for (int step = 1; step < maxS; step *= 2) {
        Level L{};
        L.off = (int)h->elims.size();
        for (auto& md : h->mem) {
            for (int j = step; j < md.nslab; j += 2 * step) {
                ElimDev E{md.slab0 + j, md.slab0 + j - step, j + step < md.nslab ? md.slab0 + j + step : -1};
                h->elims.push_back(E);
            }
        }
        L.count = (int)h->elims.size() - L.off;
        h->levels.push_back(L);
    }
    {
        Level L{};
        L.off = (int)h->elims.size();
        for (auto& md : h->mem) h->elims.push_back(ElimDev{md.slab0, -1, -1});
        L.count = (int)h->elims.size() - L.off;
        h->levels.push_back(L);
    }
    const size_t nsl = h->slabs.size();
    IfPtrs& I = h->I;
    const int NB = h->nbasis_max;
    I.NB = NB;
    I.status = h->d_status;
    I.npad = npad;
    I.xch = xch;
    I.elim_cw = elim_cw;
    if ((e = dalloc(h, &I.Gv, (size_t)h->nif * 2 * NB))) return e;
    if ((e = dalloc(h, &I.Gc, (size_t)h->nif * 2))) return e;
    if ((e = dalloc(h, &I.Gn, (size_t)h->nif * 2))) return e;
    if ((e = dalloc(h, &I.rhs, h->nif))) return e;
    if ((e = dalloc(h, &I.R, h->nif))) return e;
    if ((e = dalloc(h, &I.Cs, h->nif))) return e;
    if ((e = dalloc(h, &I.colmax, h->nif))) return e;
    if ((e = dalloc(h, &I.x, h->nif))) return e;
    if ((e = dalloc(h, &I.r, h->nif))) return e;
    if ((e = dalloc(h, &I.bq, h->nif))) return e;
    if ((e = dalloc(h, &I.D, (size_t)offD))) return e;
    if ((e = dalloc(h, &I.Dinv, (size_t)offD))) return e;
    if ((e = dalloc(h, &I.Cup, (size_t)offC))) return e;
    I.Cdn = I.Cup;
    if ((e = dalloc(h, &I.Rup, (size_t)offR))) return e;
    I.Rdn = I.Rup;
    if ((e = dalloc(h, &I.idx, idxpool.size()))) return e;
    if ((e = dalloc(h, &I.rnorm, 2 * nmem))) return e;
    if ((e = dalloc(h, &h->d_slabs, nsl))) return e;
    if ((e = dalloc(h, &h->d_elims, h->elims.size()))) return e;
    if ((e = dalloc(h, &h->d_row_member, h->nif))) return e;

    I.slabs = h->d_slabs;
    CUDA_TRY(h, cudaMemcpyAsync(I.idx, idxpool.data(), sizeof(int) * idxpool.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_slabs, h->slabs.data(), sizeof(SlabDev) * nsl, cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_elims, h->elims.data(), sizeof(ElimDev) * h->elims.size(),
                                cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_row_member, row_member.data(), sizeof(int) * h->nif,
                                cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    return 0;
}

static int check_status(mrcm_handle* h) {
    int st[MRCM_STATUS_WORDS];
    CUDA_TRY(h, cudaMemcpyAsync(st, h->d_status, sizeof(int) * MRCM_STATUS_WORDS, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->loc_ir = std::max(h->loc_ir, st[1]);
    if (st[0] & ST_NOT_SPD) return fail(h, MRCM_ERR_NOT_SPD, "non-positive pivot in a local factorisation (item " + std::to_string(st[2]) + ")");
    if (st[0] & ST_NO_CONV) return fail(h, MRCM_ERR_NO_CONVERGENCE, "local iterative refinement did not reach ir_tol");
    if (st[0] & ST_BAD) return fail(h, MRCM_ERR_TIMEOUT, "a staged copy did not complete within its wait limit");
    if (st[0] & ST_CHECK) {
        const long long v = (long long)(unsigned)st[6] | ((long long)st[7] << 32);
        return fail(h, MRCM_ERR_CHECK, "bounds check failed at site " + std::to_string(st[4]) + " (block " +
                                           std::to_string(st[5]) + ", value " + std::to_string(v) + ")");
    }
    return 0;
}

// Internal accessors for the output path that lives with its static scratch (state.cu).
int mrcm_internal_member_state(mrcm_handle* h, int member, cudaStream_t* st, const double** p, const double** u,
                               long long* nc, int* nside, int* gauge, int* device) {
    if (h->stage != ST_SOLVED) return fail(h, MRCM_ERR_STATE, "no solution yet");
    *device = h->device;
    if (member < 0 || member >= (int)h->mem.size()) return fail(h, MRCM_ERR_BAD_INPUT, "bad member");
    const MemberDev& md = h->mem[member];
    *st = h->stream;
    *nside = 2 * h->dim;
    *nc = (long long)md.n[0] * md.n[1] * md.n[2];
    *p = h->d_p + md.cell_off;
    *u = h->d_u + md.cell_off * (*nside);
    *gauge = md.pure_neumann;
    return 0;
}

int mrcm_internal_fail(mrcm_handle* h, int code, const char* msg) { return fail(h, code, msg); }

// ---------------------------------------------------------------------------
// kernel-issuing pieces of the pipeline (no host synchronisation inside)
// ---------------------------------------------------------------------------
static int issue_basis(mrcm_handle* h) {
    Phase ph(h, 0);
    // 2D: the classes write disjoint outputs and keep no per-CTA scratch in
    // global memory: the largest on the handle's stream, the others on their
    // own streams, so that their CTAs fill the SMs the largest class's last
    // wave leaves idle (3D classes share the iterate scratch indexed by the
    // CTA: one after the other)
    const size_t nc = h->jclasses.size();
    const bool concurrent = h->dim == 2 && nc > 1;
    std::vector<size_t> order(nc);
    for (size_t k = 0; k < nc; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const double wa = (double)h->jclasses[a].count * h->jclasses[a].smem;
        const double wb = (double)h->jclasses[b].count * h->jclasses[b].smem;
        return wa > wb;
    });
    if (concurrent) {
        while (h->class_streams.size() < nc - 1) {
            cudaStream_t cs = nullptr;
            CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            h->class_streams.push_back(cs);
        }
        while (h->class_events.size() < nc) {
            cudaEvent_t ev = nullptr;
            CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            h->class_events.push_back(ev);
        }
        CUDA_TRY(h, cudaEventRecord(h->class_events[0], h->stream));
        for (size_t k = 0; k + 1 < nc; ++k) CUDA_TRY(h, cudaStreamWaitEvent(h->class_streams[k], h->class_events[0], 0));
    }
    for (size_t r = 0; r < nc; ++r) {
        const JobClass& jc = h->jclasses[order[r]];
        cudaStream_t st = (r == 0 || !concurrent) ? h->stream : h->class_streams[r - 1];
        cudaError_t e = h->dim == 3 ? launch_local3d(h->P, h->mth, h->d_jobs + jc.off, jc.count, jc.smem, st)
                                    : launch_local2d(h->P, h->mth, h->d_jobs + jc.off, jc.count, jc.bw, jc.smem, st);
        if (e != cudaSuccess) return fail(h, MRCM_ERR_CUDA, std::string("local kernel: ") + cudaGetErrorString(e));
        h->launches[0] += 1;
    }
    for (size_t k = 0; concurrent && k + 1 < nc; ++k) {
        CUDA_TRY(h, cudaEventRecord(h->class_events[1 + k], h->class_streams[k]));
        CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->class_events[1 + k], 0));
    }
    return 0;
}

static int issue_interface_factor(mrcm_handle* h) {
    cudaStream_t st = h->stream;
    IfPtrs& I = h->I;
    Phase ph(h, 1);
    CUDA_TRY(h, if_assemble(h->P, h->mth, I, (int)h->sub.size(), h->nif, st));
    CUDA_TRY(h, bcr_fill(I, (int)h->slabs.size(), st));
    h->launches[1] += 4;
    for (size_t l = 0; l < h->levels.size(); ++l) {
        Level& L = h->levels[l];
        if (L.count == 0) continue;
        {
            Phase lu(h, 6);
            CUDA_TRY(h, lu_inverse(I, h->d_elims + L.off, L.count, h->d_status, h->slab_variant, st));
        }
        h->launches[1] += 1;
        h->launches[6] += 1;
        if (l + 1 < h->levels.size()) {
            CUDA_TRY(h, bcr_elim(I, h->d_elims + L.off, L.count, h->elim_smem, st));
            h->launches[1] += 1;
        }
    }
    return 0;
}

static int issue_residual(mrcm_handle* h) {
    Phase ph(h, 2);
    CUDA_TRY(h, cudaMemsetAsync(h->I.rnorm, 0, sizeof(unsigned long long) * 2 * h->mem.size(), h->stream));
    CUDA_TRY(h, if_residual(h->I, h->d_row_member, h->nif, 1, h->stream));
    h->launches[2] += 1;
    return 0;
}

// the FP32 block-cyclic-reduction sweeps on I.bq, in place
static int issue_bcr_sweeps(mrcm_handle* h) {
    const int nlev = (int)h->levels.size();
    for (int l = 0; l < nlev; ++l) {
        const Level& L = h->levels[l];
        CUDA_TRY(h, bcr_fwd(h->I, h->d_elims + L.off, L.count, h->npad, h->stream));
        h->launches[2] += 1;
    }
    for (int l = nlev - 2; l >= 0; --l) {
        const Level& L = h->levels[l];
        CUDA_TRY(h, bcr_bwd(h->I, h->d_elims + L.off, L.count, h->npad, h->stream));
        h->launches[2] += 1;
    }
    return 0;
}

static int issue_if_sweeps(mrcm_handle* h) {
    Phase ph(h, 2);
    const int nlev = (int)h->levels.size();
    for (int l = 0; l < nlev; ++l) {
        const Level& L = h->levels[l];
        CUDA_TRY(h, bcr_fwd(h->I, h->d_elims + L.off, L.count, h->npad, h->stream));
        h->launches[2] += 1;
    }
    for (int l = nlev - 2; l >= 0; --l) {
        const Level& L = h->levels[l];
        CUDA_TRY(h, bcr_bwd(h->I, h->d_elims + L.off, L.count, h->npad, h->stream));
        h->launches[2] += 1;
    }
    CUDA_TRY(h, if_update(h->I, h->nif, h->stream));
    h->launches[2] += 1;
    return 0;
}

// worst relative residual over the members (synchronises)
static int read_if_residual(mrcm_handle* h, double* worst) {
    const int nmem = (int)h->mem.size();
    std::vector<unsigned long long> nrm(2 * nmem);
    CUDA_TRY(h, cudaMemcpyAsync(nrm.data(), h->I.rnorm, sizeof(unsigned long long) * 2 * nmem,
                                cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    double w = 0.0;
    for (int m = 0; m < nmem; ++m) {
        double rn, bn;
        std::memcpy(&rn, &nrm[2 * m], 8);
        std::memcpy(&bn, &nrm[2 * m + 1], 8);
        const double r = bn > 0 ? rn / bn : rn;
        if (!(r <= w)) w = r;   // a NaN residual stays NaN (and is caught as a divergence)
    }
    *worst = w;
    return 0;
}

static int issue_assemble(mrcm_handle* h) {
    Phase ph(h, 3);
    CUDA_TRY(h, h->dim == 3 ? launch_assemble3d(h->P, h->I.x, (int)h->sub.size(), h->ncell_i_max, h->stream)
                            : launch_assemble2d(h->P, h->I.x, (int)h->sub.size(), h->ncell_i_max, h->stream));
    h->launches[3] += 1;
    return 0;
}

static int issue_smooth(mrcm_handle* h, int n_steps) {
    const int nc = 1 << h->dim;
    Phase ph(h, 4);
    for (int k = 0; k < n_steps; ++k) {
        for (int c = 0; c < nc; ++c) {
            const int off = h->colour_off[c], cnt = h->colour_off[c + 1] - off;
            cudaError_t e = h->dim == 3
                                ? launch_smooth3d(h->P, h->mth, h->d_colour_items + off, cnt, h->smooth_smem, h->stream)
                                : launch_smooth2d(h->P, h->mth, h->d_colour_items + off, cnt, h->smooth_smem, h->stream);
            if (e != cudaSuccess) return fail(h, MRCM_ERR_CUDA, std::string("smoothing kernel: ") + cudaGetErrorString(e));
            h->launches[4] += 1;
        }
    }
    h->local_solves += (long long)n_steps * h->sub.size();
    return 0;
}

// ---------------------------------------------------------------------------
// reverse pass (differentiation with respect to log K)
// ---------------------------------------------------------------------------
static int prepare_adjoint(mrcm_handle* h) {
    AdjWork& W = h->adj;
    if (W.ready) return 0;
    const int prec = h->prm.precision;
    const int nitems = (int)h->sub.size();
    const int nmem = (int)h->mem.size();
    const size_t lim = 227 * 1024;
    // jobs: basis problem on hat-Omega_i and particular problem on Omega_i,
    // grouped by band width and the number of warps that fit in shared memory
    std::map<std::pair<int, int>, std::vector<Job>> by;
    std::map<std::pair<int, int>, size_t> smem;
    for (int s = 0; s < nitems; ++s) {
        const SubDev& sd = h->sub[s];
        // (with the particular problem on hat-Omega_i the basis job carries it)
        for (int type = 0; type < (h->mth.part_hat ? 1 : 2); ++type) {
            const int nx = type == JOB_BASIS ? sd.hih[0] - sd.loh[0] : sd.hi[0] - sd.lo[0];
            const int ny = type == JOB_BASIS ? sd.hih[1] - sd.loh[1] : sd.hi[1] - sd.lo[1];
            const int bw = nx <= 8 ? 8 : nx <= 16 ? 16 : nx <= 24 ? 24 : 32;
            int nw = 4;
            while (nw > 1 && adj_local2d_smem(prec, nx, ny, nw, type == JOB_PART) > lim) nw /= 2;
            const size_t b = adj_local2d_smem(prec, nx, ny, nw, type == JOB_PART);
            if (b > lim) return fail(h, MRCM_ERR_UNSUPPORTED, "subdomain box too large for the adjoint kernels");
            by[{bw, nw}].push_back(Job{s, type});
            smem[{bw, nw}] = std::max(smem[{bw, nw}], b);
        }
        W.smooth_smem = std::max(W.smooth_smem, adj_smooth2d_smem(prec, sd.hih[0] - sd.loh[0], sd.hih[1] - sd.loh[1]));
    }
    if (W.smooth_smem > lim) return fail(h, MRCM_ERR_UNSUPPORTED, "subdomain box too large for the adjoint kernels");
    std::vector<Job> jobs;
    W.classes.clear();
    for (auto& kv : by) {
        W.classes.push_back(AdjClass{kv.first.first, kv.first.second, smem[kv.first], (int)jobs.size(),
                                     (int)kv.second.size()});
        jobs.insert(jobs.end(), kv.second.begin(), kv.second.end());
    }
    std::vector<int> col_item(std::max(h->nif, 1), 0);
    for (int s = 0; s < nitems; ++s)
        for (int k = 0; k < h->sub[s].nbasis; ++k) col_item[h->sub[s].col0 + k] = s;
    const int nside = 2 * h->dim;
    AdjPtrs& A = W.A;
    int e = 0;
    if ((e = dalloc(h, &A.gp, h->ncells))) return e;
    if ((e = dalloc(h, &A.gu, h->ncells * nside))) return e;
    if ((e = dalloc(h, &A.gTf, h->ncells * 3))) return e;
    if ((e = dalloc(h, &A.ghk, h->ncells * 3))) return e;
    if ((e = dalloc(h, &A.gwh, h->ncells * 3))) return e;
    if ((e = dalloc(h, &A.gps, (size_t)nitems * h->ncell_i_max))) return e;
    if ((e = dalloc(h, &A.gug, (size_t)nitems * MRCM_MAXSIDE * h->side_max))) return e;
    if ((e = dalloc(h, &A.gX, h->nif))) return e;
    if ((e = dalloc(h, &A.y, h->nif))) return e;
    if ((e = dalloc(h, &A.gmom, (size_t)nitems * (h->nbasis_max + 1) * MRCM_MAXSIDE * h->npsi * 2))) return e;
    if ((e = dalloc(h, &W.col_item, col_item.size()))) return e;
    if ((e = dalloc(h, &W.jobs, jobs.size()))) return e;
    if ((e = dalloc(h, &W.gout, h->ncells))) return e;
    A.X = h->I.x;
    CUDA_TRY(h, cudaMemcpyAsync(W.col_item, col_item.data(), sizeof(int) * col_item.size(), cudaMemcpyHostToDevice,
                                h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(W.jobs, jobs.data(), sizeof(Job) * jobs.size(), cudaMemcpyHostToDevice, h->stream));
    (void)nmem;
    W.ready = true;
    return 0;
}

// dL/drhs = G^-T dL/dX by refinement with the transposed slab factors.
static int solve_interface_T(mrcm_handle* h) {
    AdjWork& W = h->adj;
    cudaStream_t st = h->stream;
    const IfPtrs& I = h->I;
    const int nlev = (int)h->levels.size();
    const int max_it = std::max(8, h->prm.max_ir);
    double worst = 0.0;
    std::string hist;
    CUDA_TRY(h, cudaMemsetAsync(W.A.y, 0, sizeof(double) * h->nif, st));
    for (int it = 0;; ++it) {
        {
            Phase ph(h, 2);
            CUDA_TRY(h, cudaMemsetAsync(I.rnorm, 0, sizeof(unsigned long long) * 2 * h->mem.size(), st));
            CUDA_TRY(h, if_residualT(I, h->d_sub, W.col_item, W.A.gX, W.A.y, h->d_row_member, h->nif, 1, st));
            h->launches[2] += 1;
        }
        if (it > 0) {
            int rc = read_if_residual(h, &worst);
            if (rc) return rc;
            char buf[32];
            snprintf(buf, sizeof(buf), " %.2e", worst);
            hist += buf;
            if (!std::isfinite(worst)) return fail(h, MRCM_ERR_SINGULAR, "transposed interface refinement diverged");
            if (worst <= h->mth.ir_tol || it >= max_it) break;
        }
        Phase ph(h, 2);
        for (int l = 0; l + 1 < nlev; ++l) {
            const Level& L = h->levels[l];
            CUDA_TRY(h, bcr_bwdT(I, h->d_elims + L.off, L.count, h->npad, 0, st));
            CUDA_TRY(h, bcr_bwdT(I, h->d_elims + L.off, L.count, h->npad, 1, st));
            h->launches[2] += 2;
        }
        for (int l = nlev - 1; l >= 0; --l) {
            const Level& L = h->levels[l];
            CUDA_TRY(h, bcr_fwdT(I, h->d_elims + L.off, L.count, h->npad, st));
            h->launches[2] += 1;
        }
        CUDA_TRY(h, if_updateT(I, W.A.y, h->nif, st));
        h->launches[2] += 1;
    }
    if (worst > h->mth.ir_tol * 1e3)
        return fail(h, MRCM_ERR_NO_CONVERGENCE, "transposed interface refinement stalled; residuals:" + hist);
    return 0;
}

// Per-call metrics: with the environment variable MRCM_METRICS naming a file
// (or "stderr"), every outermost call of the solve path appends one JSON line
// with its host wall time, return code, the refinement counts and residual,
// and the slab-inverse choice of the autotuner.
static const char* const kSlabNamesLog[3] = {"gauss-jordan", "lu", "gauss-jordan-registers"};

struct CallLog {
    mrcm_handle* h;
    const char* name;
    const int* rc;
    std::chrono::steady_clock::time_point t0;
    CallLog(mrcm_handle* hh, const char* nm, const int* r) : h(hh), name(nm), rc(r), t0(std::chrono::steady_clock::now()) {
        ++h->call_depth;
    }
    ~CallLog() {
        if (--h->call_depth > 0) return;
        const char* path = std::getenv("MRCM_METRICS");
        if (!path || !*path) return;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        const int v = h->slab_variant;
        char buf[768];
        snprintf(buf, sizeof(buf),
                 "{\"call\": \"%s\", \"rc\": %d, \"wall_ms\": %.4f, \"subdomains\": %zu, \"interface_unknowns\": %d, "
                 "\"interface_ir_steps\": %d, \"interface_residual\": %.3e, \"interface_gmres\": %s, "
                 "\"local_ir_steps_max\": %d, \"local_solves\": %lld, \"smooth_steps\": %d, \"slab_inverse\": \"%s\", "
                 "\"slab_inverse_source\": \"%s\", \"tune_ms\": {\"gauss-jordan\": %.4f, \"lu\": %.4f, "
                 "\"gauss-jordan-registers\": %.4f}}\n",
                 name, *rc, ms, h->sub.size(), h->nif, h->if_iters, h->if_res, h->if_krylov ? "true" : "false",
                 h->loc_ir, h->local_solves, h->smooth_steps, v >= 0 && v < 3 ? kSlabNamesLog[v] : "none",
                 h->tune_source == 1 ? "cache" : h->tune_source == 2 ? "measured" : "fixed", h->tune_ms[0],
                 h->tune_ms[1], h->tune_ms[2]);
        static std::mutex mu;
        std::lock_guard<std::mutex> lock(mu);
        if (std::strcmp(path, "stderr") == 0) {
            std::fputs(buf, stderr);
        } else if (FILE* f = std::fopen(path, "a")) {
            std::fputs(buf, f);
            std::fclose(f);
        }
    }
};

extern "C" {

int mrcm_create(const mrcm_grid* grid, const double* K, const double* f, const mrcm_bc* bc,
                const mrcm_partition* part, const mrcm_params* params, int device_ptrs, void* cuda_stream,
                mrcm_handle** out) {
    const double* Ks[1] = {K};
    const double* fs[1] = {f};
    return create_impl(1, grid, Ks, fs, bc, part, params, device_ptrs, cuda_stream, out);
}

int mrcm_create_batch(int count, const mrcm_grid* grids, const double* const* K, const double* const* f,
                      const mrcm_bc* bcs, const mrcm_partition* parts, const mrcm_params* params,
                      int device_ptrs, void* cuda_stream, mrcm_handle** out) {
    return create_impl(count, grids, K, f, bcs, parts, params, device_ptrs, cuda_stream, out);
}

static int build_basis_body(mrcm_handle* h) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    h->err.clear();
    h->stage = ST_CREATED;
    int rc = issue_basis(h);
    if (rc) return rc;
    rc = check_status(h);
    if (rc) return rc;
    for (auto& sd : h->sub) h->local_solves += sd.nbasis + 1;
    h->stage = ST_BASIS;
    return 0;
}

int mrcm_build_basis(mrcm_handle* h) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    int rc = 0;
    CallLog log(h, "mrcm_build_basis", &rc);
    rc = build_basis_body(h);
    return rc;
}

// The interface refinement's target (relative, row-equilibrated max norm).
static double if_target(const mrcm_handle* h) { return h->mth.ir_tol; }

// Interface fallback when the refinement stalls: restarted GMRES in FP64 on
// G X = rhs, right-preconditioned by the FP32 reduction (the row scaling, the
// sweeps and the column scaling of one refinement step), started from the
// refined iterate.  G v is the residual kernel with x = v and a zero
// right-hand side (it returns -G v).  Arnoldi by classical Gram-Schmidt
// applied twice (all projections of a pass in one launch).  Dot products:
// per-block partial sums added on the host in a fixed order.  Ends when the library's residual test
// (worst member, max norm relative to the right-hand side) reaches ir_tol.
static int krylov_interface(mrcm_handle* h, double* worst_out) {
    const int n = h->nif, m = 30, max_restarts = 20;
    cudaStream_t st = h->stream;
    const int nb = kry_blocks();
    if (!h->d_kry) {
        if (int e = dalloc(h, &h->d_kry, (size_t)(m + 4) * n + (size_t)(m + 1) * nb)) return e;
    }
    double* V = h->d_kry;                    // (m + 1) x n Krylov basis
    double* w = V + (size_t)(m + 1) * n;     // n
    double* u = w + n;                       // n
    double* zero = u + n;                    // n (zero right-hand side)
    double* part = zero + n;                 // (m + 1) x nb partial sums
    CUDA_TRY(h, cudaMemsetAsync(zero, 0, sizeof(double) * n, st));
    std::vector<double> hp(nb);
    double rhs2 = 0.0;
    auto dot = [&](const double* a, const double* b, double* out) -> int {
        CUDA_TRY(h, kry_dot(a, b, n, part, st));
        CUDA_TRY(h, cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(h, cudaStreamSynchronize(st));
        double acc = 0.0;
        for (int i = 0; i < nb; ++i) acc += hp[i];
        *out = acc;
        return 0;
    };
    // hv[i] = v_i . w for the nv vectors of V (one launch, one read back)
    std::vector<double> hpm;
    auto mdot = [&](const double* Vb, const double* wv, int nv, double* out) -> int {
        hpm.resize((size_t)nv * nb);
        CUDA_TRY(h, kry_mdot(Vb, wv, n, nv, part, st));
        CUDA_TRY(h, cudaMemcpyAsync(hpm.data(), part, sizeof(double) * nv * nb, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(h, cudaStreamSynchronize(st));
        for (int i = 0; i < nv; ++i) {
            double acc = 0.0;
            for (int b = 0; b < nb; ++b) acc += hpm[(size_t)i * nb + b];
            out[i] = acc;
        }
        return 0;
    };
    // z = M^-1 v (through I.bq)
    auto precond = [&](const double* v, double* z) -> int {
        CUDA_TRY(h, kry_to_bq(h->I, v, n, st));
        if (int e = issue_bcr_sweeps(h)) return e;
        CUDA_TRY(h, kry_from_bq(h->I, z, n, st));
        return 0;
    };
    if (int e = dot(h->I.rhs, h->I.rhs, &rhs2)) return e;
    // the inner test, on the 2-norm, with a margin for the max-norm test that ends a cycle
    const double target = 1e-2 * if_target(h) * std::sqrt(rhs2);
    IfPtrs J = h->I;   // G v: x = v, rhs = 0, result (-G v) into w
    J.rhs = zero;
    J.r = w;
    double worst = 0.0;
    for (int rs = 0; rs < max_restarts; ++rs) {
        // r0 = rhs - G x into I.r; beta = |r0|
        if (int e = issue_residual(h)) return e;
        if (int e = read_if_residual(h, &worst)) return e;
        if (!std::isfinite(worst)) return fail(h, MRCM_ERR_SINGULAR, "interface Krylov iteration diverged");
        if (worst <= if_target(h)) break;
        double beta2 = 0.0;
        if (int e = dot(h->I.r, h->I.r, &beta2)) return e;
        const double beta = std::sqrt(beta2);
        if (beta == 0.0) break;
        CUDA_TRY(h, kry_axpby(V, h->I.r, 1.0 / beta, 0.0, n, st));
        std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0);
        g[0] = beta;
        int kk = 0;
        for (int j = 0; j < m; ++j) {
            kk = j + 1;
            if (int e = precond(V + (size_t)j * n, u)) return e;
            J.x = u;
            CUDA_TRY(h, if_residual(J, h->d_row_member, n, 0, st));   // w = -G u
            CUDA_TRY(h, kry_axpby(w, w, 0.0, -1.0, n, st));            // w = G u
            // classical Gram-Schmidt, applied twice (CGS2): each pass projects w
            // on all basis vectors in one launch and one host read
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<double> hc(j + 1, 0.0);
                if (int e = mdot(V, w, j + 1, hc.data())) return e;
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] += hc[i];
                CUDA_TRY(h, kry_msub(w, V, hc.data(), j + 1, n, st));
            }
            double hn2 = 0.0;
            if (int e = dot(w, w, &hn2)) return e;
            const double hn = std::sqrt(hn2);
            H[(size_t)(j + 1) * m + j] = hn;
            // previous rotations on column j, then a new one
            for (int i = 0; i < j; ++i) {
                const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[(size_t)j * m + j], b = hn;
            const double rr = std::sqrt(a * a + b * b);
            cs[j] = rr > 0 ? a / rr : 1.0;
            sn[j] = rr > 0 ? b / rr : 0.0;
            H[(size_t)j * m + j] = rr;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (hn == 0.0 || std::fabs(g[j + 1]) <= target) break;
            CUDA_TRY(h, kry_axpby(V + (size_t)(j + 1) * n, w, 1.0 / hn, 0.0, n, st));
        }
        // y = H^-1 g (upper triangular kk x kk); x += M^-1 (V y)
        std::vector<double> y(kk, 0.0);
        for (int i = kk - 1; i >= 0; --i) {
            double t = g[i];
            for (int k = i + 1; k < kk; ++k) t -= H[(size_t)i * m + k] * y[k];
            const double d = H[(size_t)i * m + i];
            y[i] = d != 0.0 ? t / d : 0.0;
        }
        CUDA_TRY(h, cudaMemsetAsync(w, 0, sizeof(double) * n, st));
        for (int i = 0; i < kk; ++i) CUDA_TRY(h, kry_axpby(w, V + (size_t)i * n, y[i], 1.0, n, st));
        if (int e = precond(w, u)) return e;
        CUDA_TRY(h, kry_axpby(h->I.x, u, 1.0, 1.0, n, st));
    }
    // the residual of the final iterate (also leaves I.r and the norms current)
    if (int e = issue_residual(h)) return e;
    if (int e = read_if_residual(h, &worst)) return e;
    *worst_out = worst;
    return 0;
}

// ---------------------------------------------------------------------------
// Interface factorisation + stationary FP64 refinement, and the autotuner of
// the slab inverses.
// ---------------------------------------------------------------------------
namespace {

// Device time of the kernels issued between start() and stop() (events on
// the handle's stream), summed over segments.
struct DevTimer {
    mrcm_handle* h;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> seg;
    cudaEvent_t a = nullptr;
    explicit DevTimer(mrcm_handle* hh) : h(hh) {}
    void start() {
        if (cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, h->stream);
    }
    void stop() {
        cudaEvent_t b = nullptr;
        if (a && cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(b, h->stream);
            seg.push_back({a, b});
        }
        a = nullptr;
    }
    double ms() {
        double t = 0.0;
        cudaStreamSynchronize(h->stream);
        for (auto& q : seg) {
            float f = 0.f;
            if (cudaEventElapsedTime(&f, q.first, q.second) == cudaSuccess) t += f;
        }
        return t;
    }
    ~DevTimer() {
        for (auto& q : seg) {
            cudaEventDestroy(q.first);
            cudaEventDestroy(q.second);
        }
        if (a) cudaEventDestroy(a);
    }
};

struct RefineOut {
    int it = 0;
    double worst = 0.0;
    bool stalled = false;
    double ms = 0.0;   // device time of the factorisation and the refinement steps
};

}  // namespace

// One factorisation with the handle's slab inverses and the refinement from
// X = 0 (residual read back after every step; stops at ir_tol, at the step
// limit, or when a step no longer reduces the residual below 0.9 of the
// previous one: then the FP32 factors are too poor a preconditioner for
// stationary refinement of this system).
static int factor_refine(mrcm_handle* h, RefineOut* o, std::string* hist) {
    DevTimer tm(h);
    tm.start();
    int rc = issue_interface_factor(h);
    if (rc) return rc;
    cudaStream_t st = h->stream;
    const int max_it = std::max(8, h->prm.max_ir);
    CUDA_TRY(h, cudaMemsetAsync(h->I.x, 0, sizeof(double) * h->nif, st));
    double prev = 0.0;
    o->stalled = false;
    o->worst = 0.0;
    int it = 0;
    for (;; ++it) {
        rc = issue_residual(h);
        if (rc) return rc;
        tm.stop();
        if (it > 0) {
            rc = read_if_residual(h, &o->worst);
            if (rc) return rc;
            char buf[32];
            snprintf(buf, sizeof(buf), " %.2e", o->worst);
            *hist += buf;
            if (!std::isfinite(o->worst)) return fail(h, MRCM_ERR_SINGULAR, "interface refinement diverged");
            if (o->worst <= if_target(h) || it >= max_it) break;
            if (it >= 2 && o->worst > 0.9 * prev) {
                o->stalled = true;
                break;
            }
            prev = o->worst;
        }
        tm.start();
        rc = issue_if_sweeps(h);
        if (rc) return rc;
    }
    o->it = it;
    o->ms = tm.ms();
    return 0;
}

// The autotuner's cache (environment MRCM_TUNE_CACHE = a JSON file): one
// object per shape class of the interface reduction, keyed by tune_key,
// holding the chosen slab inverses and the measured device times of the
// variants tried (factorisation + refinement to ir_tol; 0 when not tried).
static const char* const kSlabNames[3] = {"gauss-jordan", "lu", "gauss-jordan-registers"};

static std::string tune_key(const mrcm_handle* h) {
    char buf[192];
    snprintf(buf, sizeof(buf), "interface dim%d npad%d slabs%zu levels%zu members%zu prec%d space%d tol%.0e", h->dim,
             h->npad, h->slabs.size(), h->levels.size(), h->mem.size(), h->prm.precision, h->prm.space,
             h->mth.ir_tol);
    return buf;
}

static int tune_cache_lookup(const std::string& key) {
    const char* path = std::getenv("MRCM_TUNE_CACHE");
    if (!path || !*path) return -1;
    FILE* f = std::fopen(path, "r");
    if (!f) return -1;
    char line[512];
    int v = -1;
    const std::string tag = "\"" + key + "\": {\"slab_inverse\": \"";
    while (std::fgets(line, sizeof(line), f)) {
        const char* q = std::strstr(line, tag.c_str());
        if (!q) continue;
        q += tag.size();
        v = -1;
        for (int c = 0; c < 3; ++c) {
            const size_t len = std::strlen(kSlabNames[c]);
            if (std::strncmp(q, kSlabNames[c], len) == 0 && q[len] == '"') v = c;
        }
    }
    std::fclose(f);
    return v;
}

static void tune_cache_store(const std::string& key, int variant, const double* ms, const int* steps) {
    const char* path = std::getenv("MRCM_TUNE_CACHE");
    if (!path || !*path) return;
    std::vector<std::string> keep;
    const std::string tag = "\"" + key + "\": ";
    if (FILE* f = std::fopen(path, "r")) {
        char line[512];
        while (std::fgets(line, sizeof(line), f)) {
            std::string l(line);
            while (!l.empty() && (l.back() == '\n' || l.back() == ',' || l.back() == ' ')) l.pop_back();
            if (l.size() < 3 || l[0] == '{' || l[0] == '}' || l.find(tag) != std::string::npos) continue;
            keep.push_back(l);
        }
        std::fclose(f);
    }
    char buf[512];
    snprintf(buf, sizeof(buf),
             "  \"%s\": {\"slab_inverse\": \"%s\", \"gauss_jordan_ms\": %.4f, \"gauss_jordan_steps\": %d, "
             "\"lu_ms\": %.4f, \"lu_steps\": %d, \"gauss_jordan_registers_ms\": %.4f, \"gauss_jordan_registers_steps\": %d}",
             key.c_str(), kSlabNames[variant], ms[0], steps[0], ms[1], steps[1], ms[2], steps[2]);
    keep.push_back(buf);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    for (size_t i = 0; i < keep.size(); ++i) std::fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

static int solve_interface_body(mrcm_handle* h) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    if (h->stage != ST_BASIS) return fail(h, MRCM_ERR_STATE, "mrcm_solve_interface must follow mrcm_build_basis");
    h->err.clear();
    std::string hist;
    RefineOut o;
    int rc = 0;
    // the slab inverses this interface system admits: register-resident
    // Gauss-Jordan (slabs of up to 768 unknowns), blocked Gauss-Jordan (up to
    // 256), and the LU (any size)
    std::vector<int> cands;
    if (slab_inverse_gjr_npad(h->npad)) cands.push_back(2);
    if (slab_inverse_gj_ok(h->npad)) cands.push_back(0);
    cands.push_back(1);
    if (h->slab_variant >= 0 && std::find(cands.begin(), cands.end(), h->slab_variant) == cands.end())
        h->slab_variant = 1;
    if (h->slab_variant < 0 && cands.size() == 1) h->slab_variant = 1;
    double lu_measured = -1.0;   // the LU's final residual when this call's tuning ran it
    if (h->slab_variant < 0) {
        // autotuner: the cached choice for this shape class, else every
        // admissible slab inverse timed on this solve (device time of the
        // factorisation and the refinement steps) and the fastest one that
        // converges kept (the LU when none does)
        const std::string key = tune_key(h);
        const int cached = tune_cache_lookup(key);
        if (cached >= 0 && std::find(cands.begin(), cands.end(), cached) != cands.end()) {
            h->slab_variant = cached;
            h->tune_source = 1;
        } else {
            RefineOut run[3];
            bool ok[3] = {false, false, false};
            int steps[3] = {0, 0, 0};
            for (int c : cands) {
                h->slab_variant = c;
                hist += std::string(" [") + kSlabNames[c] + "]";
                if ((rc = factor_refine(h, &run[c], &hist))) {
                    if (rc != MRCM_ERR_SINGULAR) return rc;
                    // this variant's refinement diverged: a candidate that lost
                    run[c].worst = INFINITY;
                    h->err.clear();
                    rc = 0;
                }
                ok[c] = run[c].worst <= if_target(h);
                h->tune_ms[c] = run[c].ms;
                steps[c] = run[c].it;
            }
            // the fastest that converges; when none does, the one that got
            // closest (the GMRES fallback continues from its iterate)
            int choice = 1;
            for (int c : cands)
                if (ok[c] && (!ok[choice] || run[c].ms < run[choice].ms)) choice = c;
            if (!ok[choice])
                for (int c : cands)
                    if (std::isfinite(run[c].worst) && !(run[c].worst >= run[choice].worst)) choice = c;
            h->tune_source = 2;
            lu_measured = run[1].worst;
            tune_cache_store(key, choice, h->tune_ms, steps);
            h->slab_variant = choice;
            if (choice == cands.back() && std::isfinite(run[choice].worst)) {
                o = run[choice];   // the handle's state is the last run's
            } else {
                hist += std::string(" [") + kSlabNames[choice] + "]";
                if ((rc = factor_refine(h, &o, &hist))) return rc;
            }
        }
    }
    if (o.it == 0) {   // not solved by the tuning runs of this call
        if ((rc = factor_refine(h, &o, &hist))) return rc;
    }
    h->if_krylov = false;
    const int max_it = std::max(8, h->prm.max_ir);
    if (o.worst > if_target(h) && (o.stalled || o.it >= max_it) && h->slab_variant != 1 &&
        !(lu_measured >= 0.0 && !(lu_measured < o.worst))) {
        // a Gauss-Jordan slab inverse may be the less accurate preconditioner on a
        // very ill-conditioned interface system: refactor with the slab LU and
        // refine again (the handle keeps the LU for its later solves and
        // captures), unless this call's tuning measured the LU no closer
        h->slab_variant = 1;
        hist += " (slab LU)";
        if ((rc = factor_refine(h, &o, &hist))) return rc;
    }
    if (o.worst > if_target(h) && (o.stalled || o.it >= max_it)) {
        double worst = o.worst;
        rc = krylov_interface(h, &worst);
        if (rc) return rc;
        o.worst = worst;
        h->if_krylov = true;
        hist += " (GMRES)";
    }
    h->if_iters = o.it;
    h->if_res = o.worst;
    if (o.worst > h->mth.ir_tol * 1e3)
        return fail(h, MRCM_ERR_NO_CONVERGENCE, "interface refinement stalled; residuals:" + hist);
    rc = issue_assemble(h);
    if (rc) return rc;
    h->smooth_steps = 0;
    h->stage = ST_SOLVED;
    return 0;
}

int mrcm_solve_interface(mrcm_handle* h) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    int rc = 0;
    CallLog log(h, "mrcm_solve_interface", &rc);
    rc = solve_interface_body(h);
    return rc;
}

static int smooth_body(mrcm_handle* h, int n_steps) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    if (h->stage != ST_SOLVED) return fail(h, MRCM_ERR_STATE, "mrcm_smooth must follow mrcm_solve_interface");
    if (n_steps < 0) return fail(h, MRCM_ERR_BAD_INPUT, "n_steps must be >= 0");
    h->err.clear();
    int rc = issue_smooth(h, n_steps);
    if (rc) return rc;
    h->smooth_steps += n_steps;
    return check_status(h);
}

int mrcm_smooth(mrcm_handle* h, int n_steps) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    int rc = 0;
    CallLog log(h, "mrcm_smooth", &rc);
    rc = smooth_body(h, n_steps);
    return rc;
}

static int run_body(mrcm_handle* h, int n_steps, int use_graph) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    if (n_steps < 0) return fail(h, MRCM_ERR_BAD_INPUT, "n_steps must be >= 0");
    h->err.clear();
    int rc;
    if (!use_graph || h->if_iters == 0 || h->if_krylov) {
        // eager: also fixes the refinement count a captured step will use; a
        // problem whose interface needed the GMRES fallback always runs eagerly
        rc = mrcm_build_basis(h);
        if (rc) return rc;
        rc = mrcm_solve_interface(h);
        if (rc) return rc;
        rc = mrcm_smooth(h, n_steps);
        if (rc || !use_graph || h->if_krylov) return rc;
    }
    cudaStream_t st = h->stream;
    if (!h->graph_exec || h->graph_steps != n_steps) {
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        const bool prof = h->prof;
        h->prof = false;  // no profiling events inside the graph
        // the eager solve's refinement count: the same inputs and no order-
        // dependent sums make the captured sequence reproduce its result (the
        // residual is still checked after every launch)
        h->graph_nit = h->if_iters;
        // capture on a private stream (the legacy default stream cannot be captured)
        if (!h->cap_stream) CUDA_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        CUDA_TRY(h, cudaStreamSynchronize(st));
        h->stream = h->cap_stream;
        st = h->cap_stream;
        CUDA_TRY(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int crc = 0;
        do {
            if (cudaMemsetAsync(h->d_status, 0, sizeof(int), st) != cudaSuccess) { crc = MRCM_ERR_CUDA; break; }
            if ((crc = issue_basis(h))) break;
            if ((crc = issue_interface_factor(h))) break;
            if (cudaMemsetAsync(h->I.x, 0, sizeof(double) * h->nif, st) != cudaSuccess) { crc = MRCM_ERR_CUDA; break; }
            for (int it = 0; it < h->graph_nit && !crc; ++it) {
                if ((crc = issue_residual(h))) break;
                crc = issue_if_sweeps(h);
            }
            if (crc) break;
            if ((crc = issue_residual(h))) break;  // residual of the final iterate, checked after the launch
            if ((crc = issue_assemble(h))) break;
            crc = issue_smooth(h, n_steps);
        } while (0);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        h->prof = prof;
        h->stream = h->user_stream;
        st = h->stream;
        if (crc) {
            if (g) cudaGraphDestroy(g);
            return crc;
        }
        if (ce != cudaSuccess) return fail(h, MRCM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&h->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(h, MRCM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        h->graph_steps = n_steps;
    }
    {
        Phase ph(h, 5);
        CUDA_TRY(h, cudaGraphLaunch(h->graph_exec, st));
    }
    h->launches[5] += 1;
    double worst = 0.0;
    rc = read_if_residual(h, &worst);
    if (rc) return rc;
    h->if_res = worst;
    if (!std::isfinite(worst) || worst > h->mth.ir_tol * 1e3)
        return fail(h, MRCM_ERR_NO_CONVERGENCE, "captured step: interface refinement count too small");
    rc = check_status(h);
    if (rc) return rc;
    h->smooth_steps = n_steps;
    h->stage = ST_SOLVED;
    return 0;
}

int mrcm_run(mrcm_handle* h, int n_steps, int use_graph) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    int rc = 0;
    CallLog log(h, "mrcm_run", &rc);
    rc = run_body(h, n_steps, use_graph);
    return rc;
}

int mrcm_fluxes(mrcm_handle* h, int member, double* u_cellfaces, double* p_cells, int device_ptrs) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    if (h->stage != ST_SOLVED) return fail(h, MRCM_ERR_STATE, "no solution yet");
    if (member < 0 || member >= (int)h->mem.size()) return fail(h, MRCM_ERR_BAD_INPUT, "bad member");
    const MemberDev& md = h->mem[member];
    long long nc = (long long)md.n[0] * md.n[1] * md.n[2];
    const int nside = 2 * h->dim;
    cudaStream_t st = h->stream;
    double *pd = p_cells, *ud = u_cellfaces;
    double *tp = nullptr, *tu = nullptr;
    if (!device_ptrs) {
        if (p_cells) CUDA_TRY(h, cudaMallocAsync((void**)&tp, sizeof(double) * nc, st));
        if (u_cellfaces) CUDA_TRY(h, cudaMallocAsync((void**)&tu, sizeof(double) * nc * nside, st));
        pd = tp;
        ud = tu;
    }
    CUDA_TRY(h, launch_output(h->d_mem, (int)h->mem.size(), member, h->d_p, h->d_u, md.cell_off, nc, nside,
                              h->d_mean, pd, ud, st));
    if (!device_ptrs) {
        if (p_cells) CUDA_TRY(h, cudaMemcpyAsync(p_cells, tp, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
        if (u_cellfaces)
            CUDA_TRY(h, cudaMemcpyAsync(u_cellfaces, tu, sizeof(double) * nc * nside, cudaMemcpyDeviceToHost, st));
        if (tp) cudaFreeAsync(tp, st);
        if (tu) cudaFreeAsync(tu, st);
        CUDA_TRY(h, cudaStreamSynchronize(st));
    }
    return 0;
}

int mrcm_set_permeability(mrcm_handle* h, const double* values, int is_log, int device_ptrs) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    if (!values) return fail(h, MRCM_ERR_BAD_INPUT, "null permeability");
    h->err.clear();
    cudaStream_t st = h->stream;
    const long long nc = h->ncells;
    if (!device_ptrs) {
        for (long long c = 0; c < nc; ++c) {
            const double v = values[c];
            if (!std::isfinite(v) || (!is_log && !(v > 0.0)))
                return fail(h, MRCM_ERR_BAD_INPUT, "K must be positive and finite");
        }
    }
    const double* src = values;
    double* tmp = nullptr;
    if (!device_ptrs) {
        CUDA_TRY(h, cudaMallocAsync((void**)&tmp, sizeof(double) * nc, st));
        CUDA_TRY(h, cudaMemcpyAsync(tmp, values, sizeof(double) * nc, cudaMemcpyHostToDevice, st));
        src = tmp;
    }
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * MRCM_STATUS_WORDS, st));
    CUDA_TRY(h, launch_set_K(src, h->d_K, nc, is_log, h->d_status, st));
    if (tmp) CUDA_TRY(h, cudaFreeAsync(tmp, st));
    long long maxc = 0;
    for (auto& md : h->mem) maxc = std::max(maxc, (long long)md.n[0] * md.n[1] * md.n[2]);
    CUDA_TRY(h, launch_faces(h->d_mem, (int)h->mem.size(), maxc, h->d_K, h->d_Tf, h->d_hk, h->d_wh, st));
    int stv = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&stv, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    h->stage = ST_CREATED;
    h->if_iters = 0;  // a captured step re-learns its refinement count
    h->slab_variant = -1;   // and the new operator its slab inverses (autotuner)
    h->tune_source = 0;
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_steps = -1;
    }
    if (stv & ST_BAD_K) return fail(h, MRCM_ERR_BAD_INPUT, "K must be positive and finite");
    return 0;
}

int mrcm_backward(mrcm_handle* h, const double* dL_du, const double* dL_dp, double* dL_dlogK) {
    return mrcm_adjoint(h, dL_dp, dL_du, dL_dlogK, 0);
}

static int adjoint_body(mrcm_handle* h, const double* gp, const double* gu, double* g_logK, int device_ptrs) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    if (!g_logK) return fail(h, MRCM_ERR_BAD_INPUT, "null output");
    if (h->stage != ST_SOLVED) return fail(h, MRCM_ERR_STATE, "mrcm_adjoint needs a solution");
    if (h->dim != 2) return fail(h, MRCM_ERR_UNSUPPORTED, "the adjoint is available for 2D problems");
    for (auto& md : h->mem)
        if (md.pure_neumann)
            return fail(h, MRCM_ERR_UNSUPPORTED, "the adjoint needs Dirichlet data on some side of every member");
    h->err.clear();
    int rc = prepare_adjoint(h);
    if (rc) return rc;
    AdjWork& W = h->adj;
    AdjPtrs& A = W.A;
    cudaStream_t st = h->stream;
    const int d = h->dim, nside = 2 * d, ncol = 1 << d;
    const int ns = h->smooth_steps;
    const size_t cells = (size_t)h->ncells;
    const size_t per_snap = cells * (1 + nside);
    const size_t need = per_snap * (size_t)ns * ncol;
    if (need > W.snap_len) {
        int e = dalloc(h, &W.snap, need);
        if (e) return e;
        W.snap_len = need;
    }
    const int nitems = (int)h->sub.size();
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * MRCM_STATUS_WORDS, st));
    // replay: the MRCM-O state again, then the smoothing steps, recording the
    // state before every colour pass (forward solves with the kept factors)
    if ((rc = issue_assemble(h))) return rc;
    for (int s = 0; s < ns; ++s)
        for (int c = 0; c < ncol; ++c) {
            double* sp = W.snap + per_snap * ((size_t)s * ncol + c);
            CUDA_TRY(h, cudaMemcpyAsync(sp, h->d_p, sizeof(double) * cells, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(h, cudaMemcpyAsync(sp + cells, h->d_u, sizeof(double) * cells * nside, cudaMemcpyDeviceToDevice,
                                        st));
            Phase ph(h, 4);
            const int off = h->colour_off[c], cnt = h->colour_off[c + 1] - off;
            CUDA_TRY(h, launch_smooth2d(h->P, h->mth, h->d_colour_items + off, cnt, h->smooth_smem, st));
            h->launches[4] += 1;
        }
    // seeds
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (gp) CUDA_TRY(h, cudaMemcpyAsync(A.gp, gp, sizeof(double) * cells, kind, st));
    else CUDA_TRY(h, cudaMemsetAsync(A.gp, 0, sizeof(double) * cells, st));
    if (gu) CUDA_TRY(h, cudaMemcpyAsync(A.gu, gu, sizeof(double) * cells * nside, kind, st));
    else CUDA_TRY(h, cudaMemsetAsync(A.gu, 0, sizeof(double) * cells * nside, st));
    CUDA_TRY(h, cudaMemsetAsync(A.gTf, 0, sizeof(double) * cells * 3, st));
    CUDA_TRY(h, cudaMemsetAsync(A.ghk, 0, sizeof(double) * cells * 3, st));
    CUDA_TRY(h, cudaMemsetAsync(A.gwh, 0, sizeof(double) * cells * 3, st));
    CUDA_TRY(h, cudaMemsetAsync(A.gmom, 0,
                                sizeof(double) * nitems * (h->nbasis_max + 1) * MRCM_MAXSIDE * h->npsi * 2, st));
    // smoothing backwards: steps and colours in reverse order
    for (int s = ns - 1; s >= 0; --s)
        for (int c = ncol - 1; c >= 0; --c) {
            const double* sp = W.snap + per_snap * ((size_t)s * ncol + c);
            A.ps = sp;
            A.us = sp + cells;
            Phase ph(h, 4);
            const int off = h->colour_off[c], cnt = h->colour_off[c + 1] - off;
            CUDA_TRY(h, launch_adj_smooth2d(h->P, h->mth, A, h->d_colour_items + off, cnt, W.smooth_smem, st));
            h->launches[4] += 1;
        }
    A.ps = A.us = nullptr;
    // superposition backwards, interface transposed, moments
    {
        Phase ph(h, 3);
        CUDA_TRY(h, launch_adj_assemble2d(h->P, A, nitems, h->ncell_i_max, st));
        h->launches[3] += 1;
    }
    if (h->nif > 0) {
        if ((rc = solve_interface_T(h))) return rc;
        Phase ph(h, 3);
        CUDA_TRY(h, launch_adj_moments(h->P, h->mth, A, nitems, st));
        h->launches[3] += 1;
    }
    // basis and particular problems backwards
    {
        Phase ph(h, 0);
        for (auto& cl : W.classes) {
            CUDA_TRY(h, launch_adj_local2d(h->P, h->mth, A, W.jobs + cl.off, cl.count, cl.bw, cl.nw, cl.smem, st));
            h->launches[0] += 1;
        }
    }
    long long maxc = 0;
    for (auto& md : h->mem) maxc = std::max(maxc, (long long)md.n[0] * md.n[1] * md.n[2]);
    double* out = device_ptrs ? g_logK : W.gout;
    CUDA_TRY(h, launch_grad_logK(h->d_mem, (int)h->mem.size(), maxc, h->d_K, h->d_Tf, h->d_hk, A, out, st));
    if (!device_ptrs)
        CUDA_TRY(h, cudaMemcpyAsync(g_logK, W.gout, sizeof(double) * cells, cudaMemcpyDeviceToHost, st));
    return check_status(h);
}

int mrcm_adjoint(mrcm_handle* h, const double* gp, const double* gu, double* g_logK, int device_ptrs) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    int rc = 0;
    CallLog log(h, "mrcm_adjoint", &rc);
    rc = adjoint_body(h, gp, gu, g_logK, device_ptrs);
    return rc;
}

int mrcm_stats(const mrcm_handle* h, int* ints, int nints, double* dbl, int ndbl) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    long long vals[8] = {(long long)h->sub.size(), h->nif, h->if_iters, h->loc_ir, h->local_solves,
                         h->slab_variant < 0 ? 1 : h->slab_variant, h->if_krylov ? 1 : 0, h->tune_source};
    for (int i = 0; i < nints && i < 8; ++i) ints[i] = (int)vals[i];
    const double dv[4] = {h->if_res, h->tune_ms[0], h->tune_ms[1], h->tune_ms[2]};
    for (int i = 0; dbl && i < ndbl && i < 4; ++i) dbl[i] = dv[i];
    return 0;
}

int mrcm_profile(mrcm_handle* h, int enable) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->prof = enable != 0;
    h->ev_rec.clear();
    h->ev_used = 0;
    for (auto& v : h->launches) v = 0;
    return 0;
}

int mrcm_timings(mrcm_handle* h, double* ms, long long* launches, int n) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (auto& r : h->ev_rec) {
        float t = 0.f;
        CUDA_TRY(h, cudaEventElapsedTime(&t, r.second.first, r.second.second));
        if (r.first >= 0 && r.first < 7) acc[r.first] += t;
    }
    for (int i = 0; i < n && i < 7; ++i) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = h->launches[i];
    }
    return 0;
}

int mrcm_destroy(mrcm_handle* h) {
    if (!h) return 0;
    if (!h->allocs.empty()) {
        if (h->stream) cudaStreamSynchronize(h->stream);
        else cudaDeviceSynchronize();
    }
    for (void* p : h->allocs) cudaFree(p);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (auto cs : h->class_streams) cudaStreamDestroy(cs);
    for (auto ev : h->class_events) cudaEventDestroy(ev);
    delete h;
    return 0;
}

const char* mrcm_last_error(const mrcm_handle* h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
