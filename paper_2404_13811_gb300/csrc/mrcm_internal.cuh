// Internal structures shared by the host orchestrator and the kernels of the
// MRCM-OS library (see include/mrcm.h for the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MRCM_MAXD 3
#define MRCM_MAXSIDE 6

// Per problem (ensemble member) data visible to kernels.
struct MemberDev {
    int dim;
    int n[3];
    double h[3];
    int bc_kind[6];
    double bc_val[6];
    int sub[3];
    int overlap;
    int M[3];          // subdomains per axis
    long long cell_off;  // first cell of this member in the concatenated cell arrays
    int sub0, nsub;    // work items (subdomains) of this member
    int if0, nif;      // interface unknowns of this member
    int pure_neumann;
    double Hw[3];      // subdomain width per axis (H in beta = alpha H / K_H)
    int slab0, nslab;  // interface slabs of this member
};

// Per subdomain (work item) data.
struct SubDev {
    int member;
    int multi[3];
    int lo[3], hi[3];      // Omega_i (cells, hi exclusive)
    int loh[3], hih[3];    // hat-Omega_i
    int side_mask;         // bit sid set when side sid of Omega_i is on Gamma_i
    int nbasis;            // N_i
    int col0;              // first interface unknown (== first owned row)
    int colour;
    int nbr[6];            // neighbour work item across each side (-1 on the domain boundary)
    int slab;              // global slab id
    int slab_pos;          // offset of this subdomain's unknowns inside its slab
};

// Interface slab (block row/column of the block-tridiagonal interface
// system, one layer of subdomains along the last axis).
struct SlabDev {
    int member;
    int n;          // unknowns (= rows) in the slab
    int col0;       // first global unknown
    int nm, nv;     // rows coupled to the next / previous slab
    int up, dn;     // original neighbour slabs (-1 if none)
    long long offD, offCup, offCdn, offRup, offRdn, offPiv, offIdx; // storage offsets
    int ldc;        // leading dimension of the coupling blocks (max slab size of the member)
};

// One block-cyclic-reduction elimination: slab `j` eliminated with current
// neighbours jm (below) and jp (above, -1 when none).
struct ElimDev {
    int j, jm, jp;
};

enum JobType { JOB_BASIS = 0, JOB_PART = 1, JOB_SFACT = 2 };

struct Job {
    int item;
    int type;
};

struct DevPtrs {
    const MemberDev* mem;
    const SubDev* sub;
    const double* K;
    const double* f;
    // face coefficients per cell, 3 per cell (axes x, y, z):
    const double* Tf;    // transmissibility of the face to the +axis neighbour (0 on the boundary)
    const double* hk;    // h_a / (2 K) of the cell
    const double* wh;    // H_a / K_H of the face to the +axis neighbour (beta = alpha * wh)
    double* p;           // state pressure [ncells total]
    double* u;           // state velocities [ncells total][2*dim]
    // factors kept for smoothing
    void* fac;           // T elements
    long long fac_stride;
    void* fac_aux;       // 3D: factor of the basis box when alpha_basis != alpha_smooth
    void* fac_part;      // 3D: factor of the Omega_i box of the particular problem
    long long part_stride;
    double* xs;          // 3D mixed form: FP64 iterates of the local solves, per CTA slot
    long long xs_stride;
    double* dsc;         // Jacobi scaling of the smoothing operator (mixed form)
    long long dsc_stride;
    double* bsrc;        // particular problem on hat-Omega_i: scratch for its right-hand side [item][dsc_stride],
                         // written and read within one kernel (null otherwise)
    // basis data
    double* Psi;         // [item][nbasis_max][ncell_i_max]
    double* Ug;          // [item][nbasis_max][2d][side_max]
    double* pbar;        // [item][ncell_i_max]
    double* ubg;         // [item][2d][side_max]
    double* mom;         // [item][nbasis_max+1][2d][npsi][2]  (flux, pressure moments)
    int nbasis_max, ncell_i_max, side_max, npsi;
    int* status;         // [0] error bits, [1] max local refinement steps, [2] bad item, [3] refinement
                         // steps, [4..7] the first failed check of the bounds-check build
};

struct MethodDev {
    int space, npsi, prec;
    double alpha_b, alpha_s;
    double ir_tol;
    int max_ir;
    int same_alpha;
    int part_hat;      // the particular problem on hat-Omega_i (one more right-hand side of the basis job)
    long long wait0;   // cycle limit of the first wait for a staged copy in the 2D smoothing kernel
};


// Device pointers of the interface system.
struct IfPtrs {
    double* Gv;    // [row][2][NB] FP64 row entries (owner block, neighbour block)
    int* Gc;       // [row][2] first column of each block
    int* Gn;       // [row][2] column count of each block
    double* rhs;   // [row]
    double* R;     // row scale
    double* Cs;    // column scale
    unsigned long long* colmax;
    double* x;     // FP64 solution
    double* r;     // FP64 residual
    float* bq;     // FP32 right-hand side / solution (global unknown order)
    float* D;      // slab diagonal blocks (column-major, npad x npad)
    float* Dinv;   // their inverses
    float* Cup;    // coupling rows to the slab above (pool shared with Cdn)
    float* Cdn;
    float* Rup;    // couplings into an eliminated slab, saved (pool shared with Rdn)
    float* Rdn;
    int* idx;      // row index lists per slab
    const SlabDev* slabs;
    unsigned long long* rnorm;   // [2 * nmember]: residual max, rhs max (bit patterns)
    int* status;   // the handle's status words (bounds-check build)
    int NB;
    int npad;
    int xch;       // inverse columns solved together by the slab LU (fits shared memory)
    int elim_cw;   // coupling columns staged together by the Schur update
};

// Device pointers of the reverse (adjoint) pass.  Seeds and results live in
// the state layout; face-coefficient adjoints in the layout of Tf / hk / wh.
struct AdjPtrs {
    double* gp;          // [ncells]       dL/dp of the current state
    double* gu;          // [ncells][2d]   dL/du
    double* gTf;         // [ncells][3]    dL/dTf
    double* ghk;         // [ncells][3]    dL/d(h / 2K)
    double* gwh;         // [ncells][3]    dL/d(H / K_H)
    const double* ps;    // state recorded before the colour pass being reversed
    const double* us;
    double* gps;         // [item][ncell_i_max]        dL/d(assembled Omega_i pressure)
    double* gug;         // [item][6][side_max]        dL/d(Gamma_i face velocity)
    double* gX;          // [nif]                      dL/dX
    double* y;           // [nif]                      G^-T dL/dX  (= dL/drhs)
    double* gmom;        // like DevPtrs::mom          dL/d(moments)
    const double* X;     // forward interface solution
};

// Bounds-check build (compiled with -DMRCM_CHECK=1 into libmrcm_check.so):
// kernels test their shared-memory layouts against the launch's dynamic
// shared memory, the addresses and sizes of their bulk copies, the pivot
// records of the slab inverses and the cell indices of their state and
// slab-block writes; the first failed check is recorded in status[4..7]
// (site, block, value low / high word), the access it guards is skipped and
// the call returns MRCM_ERR_CHECK.  Without the flag every check is the
// constant true.  Sites: 1 k_local2d layout, 2 k_smooth2d layout, 3 its pack
// copy, 4 its state writes, 5 k_assemble2d state writes, 6 k_local3d /
// k_smooth3d layout, 7 k_smooth3d / k_assemble3d-style 3D state writes,
// 8 k_bcr_fill block writes, 9 k_gjr_inverse pivot records, 10 its inverse
// writes.
#ifndef MRCM_CHECK
#define MRCM_CHECK 0
#endif
#define MRCM_STATUS_WORDS 8

__device__ __forceinline__ bool mrcm_check(int* status, bool ok, int site, long long value) {
#if MRCM_CHECK
    if (!ok && status) {
        if (atomicCAS(&status[4], 0, site) == 0) {
            status[5] = (int)blockIdx.x;
            status[6] = (int)(value & 0xffffffffLL);
            status[7] = (int)(value >> 32);
        }
        atomicOr(&status[0], 32);
    }
    return ok;
#else
    (void)status;
    (void)site;
    (void)value;
    return true;
#endif
}

__device__ __forceinline__ unsigned mrcm_dyn_smem_bytes() {
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// status bits
#define ST_NOT_SPD 1
#define ST_NO_CONV 2
#define ST_SINGULAR 4
#define ST_BAD 8         // a staged (bulk) copy did not arrive within its wait limit
#define ST_BAD_K 16      // a permeability that is not positive and finite
#define ST_CHECK 32      // a check of the bounds-check build failed (status[4..7])

static inline __host__ __device__ int side_axis(int sid) { return sid >> 1; }
