// Assembly of the MRCM-O solution from the interface coefficients and the
// kept basis data (Eqs. (addu), (addp), (uhatphat); Algorithm 1, Step 5), and
// output of the current solution.
#include "mrcm_internal.cuh"
#include <algorithm>


// One CTA per subdomain: p = pbar + sum_k X_k Psi_k on Omega_i, Gamma_i
// velocities ubar + sum_k X_k U_k, interior faces from the assembled
// pressure (the same face law holds for every term of the superposition),
// physical faces from the boundary data.
__global__ void k_assemble2d(DevPtrs P, const double* __restrict__ X) {
    extern __shared__ double ps[];
    const int item = blockIdx.x;
    const SubDev sd = P.sub[item];
    const MemberDev& md = P.mem[sd.member];
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int n = nIx * nIy;
    const double* xs = X + sd.col0;
    const double* Psi = P.Psi + (size_t)item * P.nbasis_max * P.ncell_i_max;
    const double* pb = P.pbar + (size_t)item * P.ncell_i_max;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double v = pb[c];
        for (int k = 0; k < sd.nbasis; ++k) v += xs[k] * Psi[(size_t)k * P.ncell_i_max + c];
        ps[c] = v;
    }
    __syncthreads();
    const double* K = P.K + md.cell_off;
    double* pw = P.p + md.cell_off;
    double* uw = P.u + md.cell_off * 4;
    const double hx = md.h[0], hy = md.h[1];
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int i = c % nIx, j = c / nIx;
        const int gx = sd.lo[0] + i, gy = sd.lo[1] + j;
        const long long g = gx + (long long)md.n[0] * gy;
        if (!mrcm_check(P.status, g >= 0 && g < (long long)md.n[0] * md.n[1], 5, g)) continue;
        const double pc = ps[c];
        const double kc = K[g];
        pw[g] = pc;
        for (int sid = 0; sid < 4; ++sid) {
            const int a = sid >> 1;
            const bool hi = sid & 1;
            const int li = a == 0 ? i : j;
            const int lext = a == 0 ? nIx : nIy;
            const bool edge = hi ? (li == lext - 1) : (li == 0);
            const double area = a == 0 ? hy : hx;
            const double h = a == 0 ? hx : hy;
            double uo;
            if (!edge) {
                const int cn = c + (a == 0 ? (hi ? 1 : -1) : (hi ? nIx : -nIx));
                const long long gn = g + (a == 0 ? (hi ? 1 : -1) : (hi ? md.n[0] : -md.n[0]));
                const double kn = K[gn];
                const double T = area * 2.0 * kc * (kn / (kc + kn)) / h;   // no K_L K_R product (range)
                uo = T * (pc - ps[cn]) / area;
            } else if (sd.side_mask & (1 << sid)) {
                const int e = a == 0 ? j : i;
                double v = P.ubg[((size_t)item * MRCM_MAXSIDE + sid) * P.side_max + e];
                for (int k = 0; k < sd.nbasis; ++k)
                    v += xs[k] * P.Ug[(((size_t)item * P.nbasis_max + k) * MRCM_MAXSIDE + sid) * P.side_max + e];
                uo = v;
            } else if (md.bc_kind[sid] == 1) {
                const double T = 2.0 * area * kc / h;
                uo = T * (pc - md.bc_val[sid]) / area;
            } else {
                uo = md.bc_val[sid];
            }
            uw[g * 4 + sid] = uo;
        }
    }
}

// Deterministic per-member mean of the pressure (one CTA per member).
__global__ void k_member_mean(const MemberDev* mem, const double* p, double* mean) {
    __shared__ double red[256];
    const MemberDev& md = mem[blockIdx.x];
    long long nc = (long long)md.n[0] * md.n[1] * (md.dim == 3 ? md.n[2] : 1);
    double s = 0.0;
    for (long long c = threadIdx.x; c < nc; c += blockDim.x) s += p[md.cell_off + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[blockIdx.x] = md.pure_neumann ? red[0] / (double)nc : 0.0;
}

__global__ void k_output(const double* p, const double* u, long long off, long long nc, int nside,
                         const double* mean, double* pout, double* uout) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    if (pout) pout[c] = p[off + c] - mean[0];
    if (uout)
        for (int s = 0; s < nside; ++s) uout[c * nside + s] = u[(off + c) * nside + s];
}

cudaError_t launch_assemble2d(const DevPtrs& P, const double* X, int nitems, int ncell_i_max,
                              cudaStream_t s) {
    k_assemble2d<<<nitems, 256, sizeof(double) * ncell_i_max, s>>>(P, X);
    return cudaGetLastError();
}

cudaError_t launch_output(const MemberDev* dmem, int nmem, int member, const double* p, const double* u,
                          long long off, long long nc, int nside, double* dmean, double* pout,
                          double* uout, cudaStream_t s) {
    k_member_mean<<<nmem, 256, 0, s>>>(dmem, p, dmean);
    k_output<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(p, u, off, nc, nside, dmean + member, pout, uout);
    return cudaGetLastError();
}

// Face coefficients of the cell-centred RT0 operator, once per problem:
// T = a 2 K_L K_R / (h (K_L + K_R)) to the +axis neighbour, h / (2K) per
// cell and H / K_H per face (so that a Robin face has T = a / (h/2K + alpha H/K_H)).
__global__ void k_faces(const MemberDev* mem, int nmem, const double* K, double* Tf, double* hk, double* wh) {
    const int m = blockIdx.y;
    if (m >= nmem) return;
    const MemberDev& md = mem[m];
    const long long nc = (long long)md.n[0] * md.n[1] * md.n[2];
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const long long g = md.cell_off + c;
    const int ix = (int)(c % md.n[0]);
    const int iy = (int)((c / md.n[0]) % md.n[1]);
    const int iz = (int)(c / ((long long)md.n[0] * md.n[1]));
    const int idx[3] = {ix, iy, iz};
    const long long st[3] = {1, md.n[0], (long long)md.n[0] * md.n[1]};
    const double kc = K[g];
    double vol = md.h[0] * md.h[1] * (md.dim == 3 ? md.h[2] : 1.0);
    for (int a = 0; a < 3; ++a) {
        double T = 0.0, w = 0.0, hh = 0.0;
        if (a < md.dim) {
            const double area = vol / md.h[a];
            hh = md.h[a] / (2.0 * kc);
            if (idx[a] < md.n[a] - 1) {
                const double kn = K[g + st[a]];
                // harmonic-mean laws written without the product K_L K_R, which
                // leaves the FP64 range for permeabilities beyond ~1e+-154
                T = area * 2.0 * kc * (kn / (kc + kn)) / md.h[a];
                w = md.Hw[a] * 0.5 * (1.0 / kc + 1.0 / kn);
            }
        }
        Tf[g * 3 + a] = T;
        hk[g * 3 + a] = hh;
        wh[g * 3 + a] = w;
    }
}

cudaError_t launch_faces(const MemberDev* dmem, int nmem, long long maxcells, const double* K, double* Tf,
                         double* hk, double* wh, cudaStream_t s) {
    dim3 grid((unsigned)((maxcells + 255) / 256), nmem);
    k_faces<<<grid, 256, 0, s>>>(dmem, nmem, K, Tf, hk, wh);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// mrcm_fluxes_static: the output path without any device allocation.
//
// mrcm_fluxes allocates a device staging buffer whenever it writes to host
// memory, and reduces the pure-Neumann pressure gauge into scratch owned by
// the handle.  Some callers cannot allocate device memory at the point where
// they read results -- an application whose device memory is already held
// by another framework's caching allocator, or a real-time loop in which no
// allocation may happen.  This variant writes into caller device buffers and
// does its multi-block gauge reduction in the fixed static array below
// (8 KB, held by every device that loads the library until the process
// exits).  It allocates nothing.
// ---------------------------------------------------------------------------
#include "../../include/mrcm.h"

#define MRCM_STATIC_PARTIALS 1024             // partial sums, one per block
#define MRCM_STATIC_CELLS_PER_BLOCK 4096      // cells summed by one block
#define MRCM_STATIC_MAX_CELLS ((long long)MRCM_STATIC_PARTIALS * MRCM_STATIC_CELLS_PER_BLOCK)
#define MRCM_STATIC_MAX_DEVICES 64

static __device__ __align__(256) double g_gauge_partials[MRCM_STATIC_PARTIALS];

// Block b sums the pressure of cells [b * CELLS_PER_BLOCK, (b + 1) * CELLS_PER_BLOCK)
// in a fixed order and writes (not accumulates) partials[b].
__global__ void k_gauge_partials_static(const double* __restrict__ p, long long nc, double* partials) {
    __shared__ double red[256];
    const long long c0 = (long long)blockIdx.x * MRCM_STATIC_CELLS_PER_BLOCK;
    const long long c1 = min(nc, c0 + MRCM_STATIC_CELLS_PER_BLOCK);
    double s = 0.0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) s += p[c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_output_static(const double* __restrict__ p, const double* __restrict__ u, long long nc, int nside,
                                const double* partials, int nblk, int gauge, double* pout, double* uout) {
    __shared__ double mean;
    if (threadIdx.x == 0) {
        double s = 0.0;
        if (gauge)
            for (int b = 0; b < nblk; ++b) s += partials[b];
        mean = gauge ? s / (double)nc : 0.0;
    }
    __syncthreads();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        if (pout) pout[c] = p[c] - mean;
        if (uout)
            for (int s = 0; s < nside; ++s) uout[c * nside + s] = u[c * nside + s];
    }
}

// internal accessors defined with the handle (api.cu)
int mrcm_internal_member_state(mrcm_handle* h, int member, cudaStream_t* st, const double** p, const double** u,
                               long long* nc, int* nside, int* gauge, int* device);
int mrcm_internal_fail(mrcm_handle* h, int code, const char* msg);

static double* g_partials_addr[MRCM_STATIC_MAX_DEVICES] = {nullptr};

extern "C" int mrcm_fluxes_static(mrcm_handle* h, int member, double* u_cellfaces, double* p_cells) {
    if (!h) return MRCM_ERR_BAD_INPUT;
    cudaStream_t st;
    const double *p, *u;
    long long nc;
    int nside, gauge, hdev;
    int rc = mrcm_internal_member_state(h, member, &st, &p, &u, &nc, &nside, &gauge, &hdev);
    if (rc) return rc;
    if (nc > MRCM_STATIC_MAX_CELLS)
        return mrcm_internal_fail(h, MRCM_ERR_UNSUPPORTED,
                                  "mrcm_fluxes_static: member larger than its static scratch (4194304 cells)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MRCM_STATIC_MAX_DEVICES)
        return mrcm_internal_fail(h, MRCM_ERR_CUDA, "mrcm_fluxes_static: no usable current device");
    // the address below belongs to the current device, the kernels run on the
    // handle's stream: both must be the handle's device
    if (dev != hdev)
        return mrcm_internal_fail(h, MRCM_ERR_BAD_INPUT,
                                  "mrcm_fluxes_static: the handle's device must be the current device");
    if (!g_partials_addr[dev]) {
        // once per device, with that device current: the device address of the
        // static array (every thread that races here stores the same value)
        void* addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_gauge_partials);
        if (e != cudaSuccess) return mrcm_internal_fail(h, MRCM_ERR_CUDA, cudaGetErrorString(e));
        g_partials_addr[dev] = (double*)addr;
    }
    double* partials = g_partials_addr[dev];
    const int nblk = (int)((nc + MRCM_STATIC_CELLS_PER_BLOCK - 1) / MRCM_STATIC_CELLS_PER_BLOCK);
    if (gauge) k_gauge_partials_static<<<nblk, 256, 0, st>>>(p, nc, partials);
    const int nout = (int)std::min<long long>((nc + 255) / 256, 4096);
    k_output_static<<<nout, 256, 0, st>>>(p, u, nc, nside, partials, nblk, gauge, p_cells, u_cellfaces);
    e = cudaGetLastError();
    if (e != cudaSuccess) return mrcm_internal_fail(h, MRCM_ERR_CUDA, cudaGetErrorString(e));
    return MRCM_OK;
}
