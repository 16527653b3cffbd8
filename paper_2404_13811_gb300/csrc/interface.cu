// Interface system of MRCM-OS (Eqs. (int_ujump)-(int_pjump); Algorithm 1,
// Steps 3 and 5) on sm_103a.
//
// Unknowns: the coefficients X^i_k of the multiscale basis of every
// subdomain.  Rows: for every coarse edge/face Gamma_ab and every test
// function psi_m of M_H (flux continuity) and V_H (pressure continuity).
// Each subdomain owns exactly N_i rows -- the flux rows of its high sides and
// the pressure rows of its low sides -- so the system is square per
// subdomain and block tridiagonal over layers ("slabs") of subdomains along
// the last axis.  It is solved by block cyclic reduction over the slabs in
// FP32 after row/column equilibration, with FP64 residuals of the unscaled
// rows driving iterative refinement to ir_tol.
#include "mrcm_internal.cuh"
#include <algorithm>


__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Step 3/4: rows of Eqs. (int_ujump)-(int_pjump) owned by each subdomain.
// ---------------------------------------------------------------------------
__global__ void k_if_assemble(DevPtrs P, MethodDev Mth, IfPtrs I, int nitems) {
    const int s = blockIdx.x;
    if (s >= nitems) return;
    const SubDev sd = P.sub[s];
    const MemberDev& md = P.mem[sd.member];
    const int npsi = Mth.npsi, NB = I.NB;
    const int d = md.dim;
    const int PS = P.nbasis_max;  // particular slot
    auto MOM = [&](int item, int slot, int sid, int m, int which) {
        return P.mom[((((size_t)item * (P.nbasis_max + 1) + slot) * MRCM_MAXSIDE + sid) * npsi + m) * 2 + which];
    };
    for (int q = threadIdx.x; q < sd.nbasis; q += blockDim.x) {
        // q -> (kind, side, m): flux rows of high sides first, then pressure rows of low sides
        int qq = q, kind = -1, sid = -1, m = 0;
        for (int a = 0; a < d && kind < 0; ++a) {
            int sh = 2 * a + 1;
            if (sd.side_mask & (1 << sh)) {
                if (qq < npsi) { kind = 0; sid = sh; m = qq; }
                else qq -= npsi;
            }
        }
        for (int a = 0; a < d && kind < 0; ++a) {
            int sl = 2 * a;
            if (sd.side_mask & (1 << sl)) {
                if (qq < npsi) { kind = 1; sid = sl; m = qq; }
                else qq -= npsi;
            }
        }
        const int row = sd.col0 + q;
        const int t = sd.nbr[sid];
        const SubDev st = P.sub[t];
        double* gv = I.Gv + (size_t)row * 2 * NB;
        double rv;
        if (kind == 0) {
            // flux continuity: sum_i (u^i . n^i, psi_m) = 0
            for (int k = 0; k < NB; ++k) gv[k] = k < sd.nbasis ? MOM(s, k, sid, m, 0) : 0.0;
            for (int k = 0; k < NB; ++k) gv[NB + k] = k < st.nbasis ? MOM(t, k, sid ^ 1, m, 0) : 0.0;
            rv = -(MOM(s, PS, sid, m, 0) + MOM(t, PS, sid ^ 1, m, 0));
        } else {
            // pressure continuity with n^i . n = +1 for the lower (t), -1 for the upper (s) subdomain
            for (int k = 0; k < NB; ++k) gv[k] = k < sd.nbasis ? -MOM(s, k, sid, m, 1) : 0.0;
            for (int k = 0; k < NB; ++k) gv[NB + k] = k < st.nbasis ? MOM(t, k, sid ^ 1, m, 1) : 0.0;
            rv = -(MOM(t, PS, sid ^ 1, m, 1) - MOM(s, PS, sid, m, 1));
        }
        if (md.pure_neumann && s == md.sub0 && q == 0) {
            // gauge X^0_0 = 0 in place of one redundant flux row
            for (int k = 0; k < 2 * NB; ++k) gv[k] = 0.0;
            gv[0] = 1.0;
            rv = 0.0;
        }
        I.Gc[2 * row] = sd.col0;
        I.Gn[2 * row] = sd.nbasis;
        I.Gc[2 * row + 1] = st.col0;
        I.Gn[2 * row + 1] = st.nbasis;
        I.rhs[row] = rv;
        double mx = 0.0;
        for (int k = 0; k < 2 * NB; ++k) mx = fmax(mx, fabs(gv[k]));
        I.R[row] = mx > 0.0 ? 1.0 / mx : 1.0;
    }
}

__global__ void k_if_colmax(IfPtrs I, int nrows) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    const double* gv = I.Gv + (size_t)row * 2 * I.NB;
    for (int b = 0; b < 2; ++b) {
        int c0 = I.Gc[2 * row + b], nc = I.Gn[2 * row + b];
        for (int k = 0; k < nc; ++k) atomic_max_pos(&I.colmax[c0 + k], fabs(I.R[row] * gv[b * I.NB + k]));
    }
}

__global__ void k_if_colscale(IfPtrs I, int ncols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double m = __longlong_as_double((long long)I.colmax[c]);
    I.Cs[c] = m > 0.0 ? 1.0 / m : 1.0;
}

// Fills the FP32 slab blocks with the equilibrated entries R G C.
__global__ void k_bcr_fill(IfPtrs I, int nslab) {
    const int j = blockIdx.x;
    if (j >= nslab) return;
    const SlabDev S = I.slabs[j];
    const int np = I.npad;
    float* D = I.D + S.offD;
    for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
        int r = t % np, c = t / np;  // column-major for the batched LU
        D[t] = (r == c && r >= S.n) ? 1.f : 0.f;
    }
    float* Cup = I.Cup + S.offCup;
    float* Cdn = I.Cdn + S.offCdn;
    for (int t = threadIdx.x; t < S.nm * S.ldc; t += blockDim.x) Cup[t] = 0.f;
    for (int t = threadIdx.x; t < S.nv * S.ldc; t += blockDim.x) Cdn[t] = 0.f;
    __syncthreads();
    const int* mpos = I.idx + S.offIdx + S.nm + S.nv;
    const int* vpos = mpos + S.n;
    const int colU = (S.up >= 0) ? I.slabs[S.up].col0 : 0;
    const int colD = (S.dn >= 0) ? I.slabs[S.dn].col0 : 0;
    for (int rr = threadIdx.x; rr < S.n; rr += blockDim.x) {
        const int row = S.col0 + rr;
        const double* gv = I.Gv + (size_t)row * 2 * I.NB;
        const double Rr = I.R[row];
        for (int b = 0; b < 2; ++b) {
            const int c0 = I.Gc[2 * row + b], nc = I.Gn[2 * row + b];
            for (int k = 0; k < nc; ++k) {
                const int c = c0 + k;
                const float v = (float)(Rr * gv[b * I.NB + k] * I.Cs[c]);
                if (c >= S.col0 && c < S.col0 + S.n) {
                    D[(size_t)(c - S.col0) * np + rr] = v;
                } else if (S.up >= 0 && c >= colU && c < colU + I.slabs[S.up].n) {
                    Cup[(size_t)mpos[rr] * S.ldc + (c - colU)] = v;
                } else if (S.dn >= 0) {
                    Cdn[(size_t)vpos[rr] * S.ldc + (c - colD)] = v;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// One block-cyclic-reduction elimination of slab j (after Dinv_j is known).
// Updates the neighbours' diagonal blocks and couplings:
//   D_jm[mrows] -= (Rup Qv) Cdn_j,  Cup_jm <- -(Rup Qm) Cup_j,
//   D_jp[vrows] -= (Rdn Qm) Cup_j,  Cdn_jp <- -(Rdn Qv) Cdn_j,
// where Qv / Qm are the columns of Dinv_j at j's pressure / flux coupling
// rows, Rup = Cup_jm (saved) and Rdn = Cdn_jp (saved).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_bcr_elim(IfPtrs I, const ElimDev* el, int nel) {
    extern __shared__ float sm[];
    const int e = blockIdx.x;
    if (e >= nel) return;
    const ElimDev E = el[e];
    const SlabDev Sj = I.slabs[E.j];
    const SlabDev Sm = I.slabs[E.jm];
    const int np = I.npad;
    const float* Dinv = I.Dinv + Sj.offD;  // column-major np x np
    const int* mrows_j = I.idx + Sj.offIdx;
    const int* vrows_j = mrows_j + Sj.nm;
    // save couplings into j
    float* Rup = I.Rup + Sj.offRup;  // nm_jm x n_j
    float* Rdn = I.Rdn + Sj.offRdn;  // nv_jp x n_j
    const float* CupM = I.Cup + Sm.offCup;
    for (int t = threadIdx.x; t < Sm.nm * Sj.n; t += blockDim.x) {
        int r = t / Sj.n, c = t % Sj.n;
        Rup[t] = CupM[(size_t)r * Sm.ldc + c];
    }
    SlabDev Sp;
    if (E.jp >= 0) {
        Sp = I.slabs[E.jp];
        const float* CdnP = I.Cdn + Sp.offCdn;
        for (int t = threadIdx.x; t < Sp.nv * Sj.n; t += blockDim.x) {
            int r = t / Sj.n, c = t % Sj.n;
            Rdn[t] = CdnP[(size_t)r * Sp.ldc + c];
        }
    }
    __syncthreads();
    // small products: A1 = Rup Qv (nm_jm x nv_j), A2 = Rup Qm (nm_jm x nm_j)
    const int nvj = Sj.nv, nmj = (E.jp >= 0) ? Sj.nm : 0;
    float* A1 = sm;                      // Sm.nm * nvj
    float* A2 = A1 + Sm.nm * nvj;        // Sm.nm * nmj
    float* A3 = A2 + Sm.nm * nmj;        // Sp.nv * nmj
    float* A4 = A3 + (E.jp >= 0 ? Sp.nv * nmj : 0);  // Sp.nv * nvj
    for (int t = threadIdx.x; t < Sm.nm * (nvj + nmj); t += blockDim.x) {
        int r = t / (nvj + nmj), q = t % (nvj + nmj);
        int col = q < nvj ? vrows_j[q] : mrows_j[q - nvj];
        const float* Q = Dinv + (size_t)col * np;  // column col of Dinv
        const float* rr = Rup + (size_t)r * Sj.n;
        float acc = 0.f;
        for (int c = 0; c < Sj.n; ++c) acc += rr[c] * Q[c];
        if (q < nvj) A1[r * nvj + q] = acc;
        else A2[r * nmj + (q - nvj)] = acc;
    }
    if (E.jp >= 0) {
        for (int t = threadIdx.x; t < Sp.nv * (nvj + nmj); t += blockDim.x) {
            int r = t / (nvj + nmj), q = t % (nvj + nmj);
            int col = q < nmj ? mrows_j[q] : vrows_j[q - nmj];
            const float* Q = Dinv + (size_t)col * np;
            const float* rr = Rdn + (size_t)r * Sj.n;
            float acc = 0.f;
            for (int c = 0; c < Sj.n; ++c) acc += rr[c] * Q[c];
            if (q < nmj) A3[r * nmj + q] = acc;
            else A4[r * nvj + (q - nmj)] = acc;
        }
    }
    __syncthreads();
    const float* Cdn_j = I.Cdn + Sj.offCdn;  // nv_j x ldc, columns = jm unknowns
    const float* Cup_j = I.Cup + Sj.offCup;  // nm_j x ldc, columns = jp unknowns
    // jm: diagonal rows and the new upper coupling
    {
        float* Dm = I.D + Sm.offD;
        float* CupM_w = I.Cup + Sm.offCup;
        const int* mrows_m = I.idx + Sm.offIdx;
        for (int t = threadIdx.x; t < Sm.nm * Sm.n; t += blockDim.x) {
            int r = t / Sm.n, c = t % Sm.n;
            float acc = 0.f;
            for (int q = 0; q < nvj; ++q) acc += A1[r * nvj + q] * Cdn_j[(size_t)q * Sj.ldc + c];
            Dm[(size_t)c * np + mrows_m[r]] -= acc;
        }
        const int njp = (E.jp >= 0) ? Sp.n : 0;
        for (int t = threadIdx.x; t < Sm.nm * Sm.ldc; t += blockDim.x) {
            int r = t / Sm.ldc, c = t % Sm.ldc;
            float acc = 0.f;
            if (c < njp)
                for (int q = 0; q < nmj; ++q) acc -= A2[r * nmj + q] * Cup_j[(size_t)q * Sj.ldc + c];
            CupM_w[t] = acc;
        }
    }
    if (E.jp >= 0) {
        float* Dp = I.D + Sp.offD;
        float* CdnP_w = I.Cdn + Sp.offCdn;
        const int* vrows_p = I.idx + Sp.offIdx + Sp.nm;
        for (int t = threadIdx.x; t < Sp.nv * Sp.n; t += blockDim.x) {
            int r = t / Sp.n, c = t % Sp.n;
            float acc = 0.f;
            for (int q = 0; q < nmj; ++q) acc += A3[r * nmj + q] * Cup_j[(size_t)q * Sj.ldc + c];
            Dp[(size_t)c * np + vrows_p[r]] -= acc;
        }
        for (int t = threadIdx.x; t < Sp.nv * Sp.ldc; t += blockDim.x) {
            int r = t / Sp.ldc, c = t % Sp.ldc;
            float acc = 0.f;
            if (c < Sm.n)
                for (int q = 0; q < nvj; ++q) acc -= A4[r * nvj + q] * Cdn_j[(size_t)q * Sj.ldc + c];
            CdnP_w[t] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Solve phase (per refinement step).
// ---------------------------------------------------------------------------
__global__ void k_if_residual(IfPtrs I, const int* row_member, int nrows, int first) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    const double* gv = I.Gv + (size_t)row * 2 * I.NB;
    double s = I.rhs[row];
    for (int b = 0; b < 2; ++b) {
        int c0 = I.Gc[2 * row + b], nc = I.Gn[2 * row + b];
        for (int k = 0; k < nc; ++k) s -= gv[b * I.NB + k] * I.x[c0 + k];
    }
    I.r[row] = s;
    I.bq[row] = (float)(I.R[row] * s);
    const int m = row_member[row];
    atomic_max_pos(&I.rnorm[2 * m], fabs(s));
    if (first) atomic_max_pos(&I.rnorm[2 * m + 1], fabs(I.rhs[row]));
}

// forward: y_j = Dinv_j b_j (stored in place), then push into the neighbours
__global__ void __launch_bounds__(256) k_bcr_fwd(IfPtrs I, const ElimDev* el, int nel) {
    extern __shared__ float y[];
    const int e = blockIdx.x;
    if (e >= nel) return;
    const ElimDev E = el[e];
    const SlabDev Sj = I.slabs[E.j];
    const int np = I.npad;
    const float* Dinv = I.Dinv + Sj.offD;
    float* bj = I.bq + Sj.col0;
    for (int r = threadIdx.x; r < Sj.n; r += blockDim.x) {
        float acc = 0.f;
        for (int c = 0; c < Sj.n; ++c) acc += Dinv[(size_t)c * np + r] * bj[c];
        y[r] = acc;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < Sj.n; r += blockDim.x) bj[r] = y[r];
    if (E.jm >= 0 && E.jm != E.j) {
        const SlabDev Sm = I.slabs[E.jm];
        const float* Rup = I.Rup + Sj.offRup;
        const int* mrows_m = I.idx + Sm.offIdx;
        float* bm = I.bq + Sm.col0;
        for (int r = threadIdx.x; r < Sm.nm; r += blockDim.x) {
            float acc = 0.f;
            for (int c = 0; c < Sj.n; ++c) acc += Rup[(size_t)r * Sj.n + c] * y[c];
            bm[mrows_m[r]] -= acc;
        }
    }
    if (E.jp >= 0) {
        const SlabDev Sp = I.slabs[E.jp];
        const float* Rdn = I.Rdn + Sj.offRdn;
        const int* vrows_p = I.idx + Sp.offIdx + Sp.nm;
        float* bp = I.bq + Sp.col0;
        for (int r = threadIdx.x; r < Sp.nv; r += blockDim.x) {
            float acc = 0.f;
            for (int c = 0; c < Sj.n; ++c) acc += Rdn[(size_t)r * Sj.n + c] * y[c];
            bp[vrows_p[r]] -= acc;
        }
    }
}

// backward: x_j = y_j - Qv (Cdn_j x_jm) - Qm (Cup_j x_jp)
__global__ void __launch_bounds__(256) k_bcr_bwd(IfPtrs I, const ElimDev* el, int nel) {
    extern __shared__ float t[];
    const int e = blockIdx.x;
    if (e >= nel) return;
    const ElimDev E = el[e];
    const SlabDev Sj = I.slabs[E.j];
    const int np = I.npad;
    const float* Dinv = I.Dinv + Sj.offD;
    const int* mrows_j = I.idx + Sj.offIdx;
    const int* vrows_j = mrows_j + Sj.nm;
    float* tv = t;             // nv
    float* tm = t + Sj.nv;     // nm
    const SlabDev Sm = I.slabs[E.jm];
    const float* Cdn_j = I.Cdn + Sj.offCdn;
    const float* Cup_j = I.Cup + Sj.offCup;
    const float* xm = I.bq + Sm.col0;
    for (int q = threadIdx.x; q < Sj.nv; q += blockDim.x) {
        float acc = 0.f;
        for (int c = 0; c < Sm.n; ++c) acc += Cdn_j[(size_t)q * Sj.ldc + c] * xm[c];
        tv[q] = acc;
    }
    const int nmj = E.jp >= 0 ? Sj.nm : 0;
    if (E.jp >= 0) {
        const SlabDev Sp = I.slabs[E.jp];
        const float* xp = I.bq + Sp.col0;
        for (int q = threadIdx.x; q < Sj.nm; q += blockDim.x) {
            float acc = 0.f;
            for (int c = 0; c < Sp.n; ++c) acc += Cup_j[(size_t)q * Sj.ldc + c] * xp[c];
            tm[q] = acc;
        }
    }
    __syncthreads();
    float* xj = I.bq + Sj.col0;
    for (int r = threadIdx.x; r < Sj.n; r += blockDim.x) {
        float acc = xj[r];
        for (int q = 0; q < Sj.nv; ++q) acc -= Dinv[(size_t)vrows_j[q] * np + r] * tv[q];
        for (int q = 0; q < nmj; ++q) acc -= Dinv[(size_t)mrows_j[q] * np + r] * tm[q];
        xj[r] = acc;
    }
}

__global__ void k_if_update(IfPtrs I, int ncols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    I.x[c] += I.Cs[c] * (double)I.bq[c];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t if_assemble(const DevPtrs& P, const MethodDev& M, const IfPtrs& I, int nitems, int nrows,
                        cudaStream_t s) {
    k_if_assemble<<<nitems, 64, 0, s>>>(P, M, I, nitems);
    cudaMemsetAsync(I.colmax, 0, sizeof(unsigned long long) * nrows, s);
    k_if_colmax<<<(nrows + 255) / 256, 256, 0, s>>>(I, nrows);
    k_if_colscale<<<(nrows + 255) / 256, 256, 0, s>>>(I, nrows);
    return cudaGetLastError();
}

cudaError_t bcr_fill(const IfPtrs& I, int nslab, cudaStream_t s) {
    k_bcr_fill<<<nslab, 256, 0, s>>>(I, nslab);
    return cudaGetLastError();
}

cudaError_t bcr_elim(const IfPtrs& I, const ElimDev* el, int nel, size_t smem, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_bcr_elim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_bcr_elim<<<nel, 512, smem, s>>>(I, el, nel);
    return cudaGetLastError();
}

cudaError_t if_residual(const IfPtrs& I, const int* row_member, int nrows, int first, cudaStream_t s) {
    k_if_residual<<<(nrows + 255) / 256, 256, 0, s>>>(I, row_member, nrows, first);
    return cudaGetLastError();
}

cudaError_t bcr_fwd(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    k_bcr_fwd<<<nel, 256, sizeof(float) * nmax, s>>>(I, el, nel);
    return cudaGetLastError();
}

cudaError_t bcr_bwd(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    k_bcr_bwd<<<nel, 256, sizeof(float) * 2 * nmax, s>>>(I, el, nel);
    return cudaGetLastError();
}

cudaError_t if_update(const IfPtrs& I, int ncols, cudaStream_t s) {
    k_if_update<<<(ncols + 255) / 256, 256, 0, s>>>(I, ncols);
    return cudaGetLastError();
}

#include <cooperative_groups.h>
namespace cg = cooperative_groups;

constexpr int GJ_NB = 32;   // panel width
constexpr int GJ_CL = 4;    // CTAs per cluster (one cluster per slab)
constexpr int GJ_THREADS = 512;

// ---------------------------------------------------------------------------
// Slab inverse through a blocked LU factorisation with partial pivoting
// (FP32, column-major np x np, in place in D, inverse written to Dinv).
// Phase 1 (cluster-synchronised per panel of GJ_NB columns): every CTA of
// the cluster factors the panel redundantly in shared memory, the owner
// writes it back, and each CTA applies the interchanges to the columns it
// owns, forms their U12 rows and updates their trailing part.
// Phase 2 (independent per CTA): the columns of the inverse owned by a CTA
// are solved from P A = L U: column j = U^-1 L^-1 e_{q(j)}.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GJ_THREADS) k_lu_inverse(IfPtrs I, const ElimDev* el, int nel, int* status) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int e = blockIdx.x / GJ_CL;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int np = I.npad;
    const int npan = (np + GJ_NB - 1) / GJ_NB;
    const int ncmax = ((npan + GJ_CL - 1) / GJ_CL) * GJ_NB;
    extern __shared__ __align__(16) float lsm[];
    float* Ps = lsm;                           // [c][r], GJ_NB * np
    float* Xs = Ps + GJ_NB * np;               // [jj][r], GJ_NB * np
    float* Upy = Xs + GJ_NB * np;              // [c][jj], GJ_NB * ncmax
    int* piv = (int*)(Upy + GJ_NB * ncmax);    // np
    int* ownc = piv + np;                      // ncmax
    int* qpos = ownc + ncmax;                  // np: position of the unit entry of P e_j
    __shared__ float redv[32];
    __shared__ int redi[32];
    __shared__ int nown;
    const bool active = e < nel;
    float* A = nullptr;
    float* Ainv = nullptr;
    if (active) {
        const SlabDev S = I.slabs[el[e].j];
        A = I.D + S.offD;
        Ainv = I.Dinv + S.offD;
    }
    if (tid == 0) {
        int c = 0;
        for (int q = rank; q < npan; q += GJ_CL)
            for (int j = q * GJ_NB; j < min(np, (q + 1) * GJ_NB); ++j) ownc[c++] = j;
        nown = c;
    }
    bool singular = false;
    // ---------------- phase 1: P A = L U ----------------
    for (int q = 0; q < npan; ++q) {
        __threadfence();
        cluster.sync();
        const int k0 = q * GJ_NB, b = min(GJ_NB, np - k0);
        if (active)
            for (int t = tid; t < b * (np - k0); t += nt) {
                int c = t / (np - k0), r = k0 + t % (np - k0);
                Ps[c * np + r] = __ldcg(&A[(size_t)(k0 + c) * np + r]);
            }
        cluster.sync();
        if (!active) continue;
        for (int c = 0; c < b; ++c) {
            const int r0 = k0 + c;
            float best = -1.f;
            int bi = r0;
            for (int r = r0 + tid; r < np; r += nt) {
                float v = fabsf(Ps[c * np + r]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o; o >>= 1) {
                float ov = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if ((tid & 31) == 0) { redv[tid >> 5] = best; redi[tid >> 5] = bi; }
            __syncthreads();
            if (tid < 32) {
                float v = tid < (nt >> 5) ? redv[tid] : -1.f;
                int ii = tid < (nt >> 5) ? redi[tid] : 0x7fffffff;
                for (int o = 16; o; o >>= 1) {
                    float ov = __shfl_xor_sync(0xffffffffu, v, o);
                    int oi = __shfl_xor_sync(0xffffffffu, ii, o);
                    if (ov > v || (ov == v && oi < ii)) { v = ov; ii = oi; }
                }
                if (tid == 0) piv[r0] = ii;
            }
            __syncthreads();
            const int p = piv[r0];
            if (p != r0)
                for (int cc = tid; cc < b; cc += nt) {
                    float t0 = Ps[cc * np + r0];
                    Ps[cc * np + r0] = Ps[cc * np + p];
                    Ps[cc * np + p] = t0;
                }
            __syncthreads();
            float a = Ps[c * np + r0];
            if (a == 0.f) { singular = true; a = 1e-30f; }
            const float ia = (float)(1.0 / (double)a);
            for (int r = r0 + 1 + tid; r < np; r += nt) Ps[c * np + r] *= ia;
            __syncthreads();
            for (int t = tid; t < (b - c - 1) * (np - r0 - 1); t += nt) {
                int cc = c + 1 + t / (np - r0 - 1), r = r0 + 1 + t % (np - r0 - 1);
                Ps[cc * np + r] -= Ps[c * np + r] * Ps[cc * np + r0];
            }
            __syncthreads();
        }
        if (q % GJ_CL == rank)
            for (int t = tid; t < b * (np - k0); t += nt) {
                int c = t / (np - k0), r = k0 + t % (np - k0);
                A[(size_t)(k0 + c) * np + r] = Ps[c * np + r];
            }
        const int no = nown;
        // interchanges on every owned column outside the panel
        for (int jj = tid; jj < no; jj += nt) {
            const int j = ownc[jj];
            if (j >= k0 && j < k0 + b) continue;
            float* col = A + (size_t)j * np;
            for (int c = 0; c < b; ++c) {
                int p = piv[k0 + c];
                if (p != k0 + c) { float t0 = col[k0 + c]; col[k0 + c] = col[p]; col[p] = t0; }
            }
        }
        __syncthreads();
        // U12 = L11^-1 A12 for owned trailing columns (one thread per column)
        for (int jj = tid; jj < no; jj += nt) {
            const int j = ownc[jj];
            if (j < k0 + b) continue;
            float* col = A + (size_t)j * np;
            float x[GJ_NB];
#pragma unroll
            for (int c = 0; c < GJ_NB; ++c) x[c] = c < b ? col[k0 + c] : 0.f;
#pragma unroll
            for (int c = 0; c < GJ_NB; ++c)
#pragma unroll
                for (int c2 = c + 1; c2 < GJ_NB; ++c2)
                    if (c2 < b) x[c2] -= Ps[c * np + k0 + c2] * x[c];
#pragma unroll
            for (int c = 0; c < GJ_NB; ++c)
                if (c < b) {
                    col[k0 + c] = x[c];
                    Upy[c * ncmax + jj] = x[c];
                }
        }
        __syncthreads();
        // trailing update A22 -= L21 U12 over owned trailing columns
        const int r1 = k0 + b;
        if (r1 < np) {
            const int ntr = (np - r1) / 4, ntc = (no + 3) / 4;
            for (int t = tid; t < ntr * ntc; t += nt) {
                const int r = r1 + (t % ntr) * 4, jj0 = (t / ntr) * 4;
                float acc[4][4];
                int jcol[4];
                bool skip[4];
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    int jj = jj0 + y;
                    jcol[y] = jj < no ? ownc[jj] : -1;
                    skip[y] = jcol[y] < r1;
#pragma unroll
                    for (int x = 0; x < 4; ++x) acc[x][y] = skip[y] ? 0.f : A[(size_t)jcol[y] * np + r + x];
                }
                for (int c = 0; c < b; ++c) {
                    const float4 s4 = *reinterpret_cast<const float4*>(&Ps[c * np + r]);
                    const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
                    float av[4];
#pragma unroll
                    for (int y = 0; y < 4; ++y) av[y] = skip[y] ? 0.f : Upy[c * ncmax + jj0 + y];
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] -= sv[x] * av[y];
                }
#pragma unroll
                for (int y = 0; y < 4; ++y)
                    if (!skip[y])
#pragma unroll
                        for (int x = 0; x < 4; ++x) A[(size_t)jcol[y] * np + r + x] = acc[x][y];
            }
        }
        __syncthreads();
    }
    __threadfence();
    cluster.sync();
    if (!active) return;
    // ---------------- phase 2: owned columns of the inverse ----------------
    if (tid == 0) {
        // rowperm[i] = original row at position i; qpos[j] = position of original row j
        int* rowperm = (int*)Upy;
        for (int i = 0; i < np; ++i) rowperm[i] = i;
        for (int c = 0; c < np; ++c) {
            int p = piv[c], t0 = rowperm[c];
            rowperm[c] = rowperm[p];
            rowperm[p] = t0;
        }
        for (int i = 0; i < np; ++i) qpos[rowperm[i]] = i;
    }
    __syncthreads();
    const int no = nown;
    for (int j0 = 0; j0 < no; j0 += GJ_NB) {
        const int nb = min(GJ_NB, no - j0);
        for (int t = tid; t < GJ_NB * np; t += nt) {
            int jj = t / np, r = t % np;
            Xs[t] = (jj < nb && r == qpos[ownc[j0 + jj]]) ? 1.f : 0.f;
        }
        __syncthreads();
        // forward with unit L, panel by panel
        for (int q = 0; q < npan; ++q) {
            const int k0 = q * GJ_NB, b = min(GJ_NB, np - k0);
            for (int t = tid; t < b * (np - k0); t += nt) {
                int c = t / (np - k0), r = k0 + t % (np - k0);
                Ps[c * np + r] = __ldcg(&A[(size_t)(k0 + c) * np + r]);
            }
            __syncthreads();
            for (int jj = tid; jj < nb; jj += nt) {
                float* xc = Xs + jj * np;
                for (int c = 0; c < b; ++c) {
                    const float xv = xc[k0 + c];
                    for (int c2 = c + 1; c2 < b; ++c2) xc[k0 + c2] -= Ps[c * np + k0 + c2] * xv;
                }
            }
            __syncthreads();
            const int r1 = k0 + b;
            for (int t = tid; t < (np - r1) * nb; t += nt) {
                int jj = t / (np - r1), r = r1 + t % (np - r1);
                float* xc = Xs + jj * np;
                float acc = xc[r];
                for (int c = 0; c < b; ++c) acc -= Ps[c * np + r] * xc[k0 + c];
                xc[r] = acc;
            }
            __syncthreads();
        }
        // backward with U, panel by panel from the last
        for (int q = npan - 1; q >= 0; --q) {
            const int k0 = q * GJ_NB, b = min(GJ_NB, np - k0);
            for (int t = tid; t < b * (k0 + b); t += nt) {
                int c = t / (k0 + b), r = t % (k0 + b);
                Ps[c * np + r] = __ldcg(&A[(size_t)(k0 + c) * np + r]);
            }
            __syncthreads();
            for (int jj = tid; jj < nb; jj += nt) {
                float* xc = Xs + jj * np;
                for (int c = b - 1; c >= 0; --c) {
                    const float xv = xc[k0 + c] / Ps[c * np + k0 + c];
                    xc[k0 + c] = xv;
                    for (int c2 = 0; c2 < c; ++c2) xc[k0 + c2] -= Ps[c * np + k0 + c2] * xv;
                }
            }
            __syncthreads();
            for (int t = tid; t < k0 * nb; t += nt) {
                int jj = t / k0, r = t % k0;
                float* xc = Xs + jj * np;
                float acc = xc[r];
                for (int c = 0; c < b; ++c) acc -= Ps[c * np + r] * xc[k0 + c];
                xc[r] = acc;
            }
            __syncthreads();
        }
        for (int t = tid; t < nb * np; t += nt) {
            int jj = t / np, r = t % np;
            Ainv[(size_t)ownc[j0 + jj] * np + r] = Xs[jj * np + r];
        }
        __syncthreads();
    }
    if (singular && tid == 0) atomicOr(status, ST_SINGULAR);
}

size_t lu_smem(int np) {
    int npan = (np + GJ_NB - 1) / GJ_NB;
    int ncmax = ((npan + GJ_CL - 1) / GJ_CL) * GJ_NB;
    size_t ncm = std::max((size_t)GJ_NB * ncmax, (size_t)np);
    return sizeof(float) * (2 * (size_t)GJ_NB * np + ncm) + sizeof(int) * ((size_t)np + ncmax + np) + 16;
}

cudaError_t lu_inverse(const IfPtrs& I, const ElimDev* el, int nel, int* status, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    size_t smem = lu_smem(I.npad);
    cudaError_t e = cudaFuncSetAttribute(k_lu_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nel * GJ_CL);
    cfg.blockDim = dim3(GJ_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = GJ_CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_lu_inverse, I, el, nel, status);
}
