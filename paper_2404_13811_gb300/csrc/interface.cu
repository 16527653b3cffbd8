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
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

constexpr int GJ_NB = 32;   // panel width
constexpr int GJ_CL = 4;    // CTAs per cluster of the Schur update (one cluster per eliminated slab)
// CTAs per cluster of the slab LU inverse (one cluster per slab): 8 when a
// launch's slabs all fit on the GPU as 8-CTA clusters at once, else 4
constexpr int LU_CL_MIN = 4, LU_CL_MAX = 8;
constexpr int GJ_THREADS = 512;
constexpr int GJ_NB_WARPS = GJ_THREADS / 32;
constexpr int PUB_PAR = GJ_NB_WARPS * GJ_NB;   // one parity of the slab LU's published panel rows
constexpr int PUB_FLOATS = 2 * PUB_PAR;        // both parities
// inverse columns solved together in phase 2: IfPtrs::xch (64 unless the
// slab is too large for shared memory)



// Programmatic dependent launch: the kernels of the refinement loop are
// launched so that each may be scheduled while its predecessor drains; each
// waits for its predecessor's completion (and memory) before touching data,
// and lets its own successor be scheduled as soon as all its CTAs run.
__device__ __forceinline__ void pdl_wait_and_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

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
                    if (mrcm_check(I.status, rr < np && c - S.col0 < np, 8, c)) D[(size_t)(c - S.col0) * np + rr] = v;
                } else if (S.up >= 0 && c >= colU && c < colU + I.slabs[S.up].n) {
                    if (mrcm_check(I.status, mpos[rr] >= 0 && mpos[rr] < S.nm && c - colU < S.ldc, 8, mpos[rr]))
                        Cup[(size_t)mpos[rr] * S.ldc + (c - colU)] = v;
                } else if (S.dn >= 0) {
                    if (mrcm_check(I.status, vpos[rr] >= 0 && vpos[rr] < S.nv && c - colD >= 0 && c - colD < S.ldc, 8,
                                   vpos[rr]))
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
// AT <- (L Q)^T with L (M x K, row-major in global memory) and Q the
// columns cols[0..N) of Dinv (rows 0..K): AT[n * Mp + m], Mp / Np = M / N
// rounded up to 4, zero beyond M / N.  K in chunks of 32 staged transposed
// (stLT[k * (Mp + 4) + m], stQ[k * (Np + 4) + n]); every thread owns 4 x 4
// output tiles, read as float4 pairs per k (16 FMAs per two loads).  The
// sum over k runs in increasing k for every entry.
__device__ void rows_times_cols(const float* L, int M, int K, const float* Dinv, int np, const int* cols, int N,
                                float* AT, float* stLT, float* stQ) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Mp = (M + 3) & ~3, Np = (N + 3) & ~3, ldl = Mp + 4, ldq = Np + 4;
    const int tm = Mp >> 2, tn = Np >> 2;
    for (int t = tid; t < Np * Mp; t += nt) AT[t] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int kb = min(32, K - k0);
        __syncthreads();
        for (int t = tid; t < Mp * 32; t += nt) {
            const int m = t >> 5, k = t & 31;
            stLT[k * ldl + m] = (k < kb && m < M) ? __ldcg(&L[(size_t)m * K + k0 + k]) : 0.f;
        }
        for (int t = tid; t < Np * 32; t += nt) {
            const int n = t >> 5, k = t & 31;
            stQ[k * ldq + n] = (k < kb && n < N) ? Dinv[(size_t)cols[n] * np + k0 + k] : 0.f;
        }
        __syncthreads();
        for (int t = tid; t < tm * tn; t += nt) {
            const int i = t / tn, jn = t - (t / tn) * tn;
            float acc[4][4];
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const float4 v = *reinterpret_cast<const float4*>(&AT[(4 * jn + y) * Mp + 4 * i]);
                acc[0][y] = v.x; acc[1][y] = v.y; acc[2][y] = v.z; acc[3][y] = v.w;
            }
            for (int k = 0; k < kb; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(&stLT[k * ldl + 4 * i]);
                const float4 q = *reinterpret_cast<const float4*>(&stQ[k * ldq + 4 * jn]);
                const float av[4] = {a.x, a.y, a.z, a.w}, qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] += av[x] * qv[y];
            }
#pragma unroll
            for (int y = 0; y < 4; ++y)
                *reinterpret_cast<float4*>(&AT[(4 * jn + y) * Mp + 4 * i]) = make_float4(acc[0][y], acc[1][y], acc[2][y], acc[3][y]);
        }
    }
    __syncthreads();
}

// Rows r < M of a target: tgt(r, c) op= sum_q A[r][q] C[q][c] for c < ncol,
// with A given transposed (AT[q * Mp + r], q < Np = M2 rounded up to 4,
// zero-padded) and C row-major (ld ldc) in global memory, staged in shared
// memory in column chunks of at most cwmax (Csm[q * cwp + c]).  4 x 4
// register tiles as above; the sum over q runs in increasing q.
template <bool ACCUM_INTO_D>
__device__ void apply_coupling(const float* AT, int M, int M2, const float* Cg, int ldc, int ncol, float* Csm,
                               int cwmax, float* D, int np, const int* rows, float* Cout, int ldout, int nclear) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Mp = (M + 3) & ~3, Np = (M2 + 3) & ~3, tm = Mp >> 2;
    for (int c0 = 0; c0 < ncol; c0 += cwmax) {
        const int cw = min(cwmax, ncol - c0), cwp = (cw + 3) & ~3, tc = cwp >> 2;
        __syncthreads();
        for (int t = tid; t < Np * cwp; t += nt) {
            const int q = t / cwp, c = t - (t / cwp) * cwp;
            Csm[t] = (q < M2 && c < cw) ? Cg[(size_t)q * ldc + c0 + c] : 0.f;
        }
        __syncthreads();
        for (int t = tid; t < tm * tc; t += nt) {
            const int i = t / tc, jc = t - (t / tc) * tc;
            float acc[4][4] = {};
            for (int q = 0; q < M2; ++q) {
                const float4 a = *reinterpret_cast<const float4*>(&AT[q * Mp + 4 * i]);
                const float4 cc = *reinterpret_cast<const float4*>(&Csm[q * cwp + 4 * jc]);
                const float av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] += av[x] * cv[y];
            }
            if (ACCUM_INTO_D) {
                // the tile's 16 entries of D read before any is written (the target
                // rows are distinct), so that the reads are in flight together
                float dv[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int r = 4 * i + x, c = 4 * jc + y;
                        dv[x][y] = (r < M && c < cw) ? D[(size_t)(c0 + c) * np + rows[r]] : 0.f;
                    }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int r = 4 * i + x, c = 4 * jc + y;
                        if (r < M && c < cw) D[(size_t)(c0 + c) * np + rows[r]] = dv[x][y] - acc[x][y];
                    }
            } else {
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const int r = 4 * i + x;
                    if (r >= M) continue;
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int c = 4 * jc + y;
                        if (c < cw) Cout[(size_t)r * ldout + c0 + c] = -acc[x][y];
                    }
                }
            }
        }
    }
    if (!ACCUM_INTO_D)
        for (int t = tid; t < M * (nclear - ncol); t += nt) {
            const int r = t / (nclear - ncol), c = ncol + t % (nclear - ncol);
            Cout[(size_t)r * ldout + c] = 0.f;
        }
}

// ---------------------------------------------------------------------------
// One block-cyclic-reduction elimination of slab j (after Dinv_j is known),
// one cluster of 4, 8 or 16 CTAs.  With Qv / Qm the columns of Dinv_j at j's
// pressure / flux coupling rows, Rup = Cup_jm and Rdn = Cdn_jp (saved first),
// CTA r computes product r mod 4 on the (r / 4)-th chunk of its rows:
//   0: D_jm[mrows] -= (Rup Qv) Cdn_j      1: Cup_jm <- -(Rup Qm) Cup_j
//   2: D_jp[vrows] -= (Rdn Qm) Cup_j      3: Cdn_jp <- -(Rdn Qv) Cdn_j
// (every target row is written by one CTA only).
// ---------------------------------------------------------------------------
constexpr int EL_THREADS = 512;

__global__ void __launch_bounds__(EL_THREADS) k_bcr_elim(IfPtrs I, const ElimDev* el, int nel) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int e = blockIdx.x / CL;
    const int prod = rank & 3, chunk = rank >> 2, nch = CL >> 2;
    extern __shared__ __align__(16) float esm[];
    const bool active = e < nel;
    ElimDev E{0, 0, -1};
    SlabDev Sj{}, Sm{}, Sp{};
    if (active) {
        E = el[e];
        Sj = I.slabs[E.j];
        Sm = I.slabs[E.jm];
        if (E.jp >= 0) Sp = I.slabs[E.jp];
    }
    const int np = I.npad;
    const int tid = threadIdx.x, nt = blockDim.x;
    float* Rup = I.Rup + Sj.offRup;  // nm_jm x n_j
    float* Rdn = I.Rdn + Sj.offRdn;  // nv_jp x n_j
    if (active) {
        // save the couplings into j (split over the cluster)
        const float* CupM = I.Cup + Sm.offCup;
        for (int t = tid + rank * nt; t < Sm.nm * Sj.n; t += nt * CL) {
            const int r = t / Sj.n, c = t - (t / Sj.n) * Sj.n;
            Rup[t] = CupM[(size_t)r * Sm.ldc + c];
        }
        if (E.jp >= 0) {
            const float* CdnP = I.Cdn + Sp.offCdn;
            for (int t = tid + rank * nt; t < Sp.nv * Sj.n; t += nt * CL) {
                const int r = t / Sj.n, c = t - (t / Sj.n) * Sj.n;
                Rdn[t] = CdnP[(size_t)r * Sp.ldc + c];
            }
        }
    }
    __threadfence();
    cluster.sync();
    if (!active) return;
    const float* Dinv = I.Dinv + Sj.offD;
    const int* mrows_j = I.idx + Sj.offIdx;
    const int* vrows_j = mrows_j + Sj.nm;
    const float* Cdn_j = I.Cdn + Sj.offCdn;  // nv_j x ldc, columns = jm unknowns
    const float* Cup_j = I.Cup + Sj.offCup;  // nm_j x ldc, columns = jp unknowns
    const bool up = prod < 2;
    if (!up && E.jp < 0) return;
    const bool useQv = (prod == 0 || prod == 3);
    const int N = useQv ? Sj.nv : Sj.nm;
    const int* cols = useQv ? vrows_j : mrows_j;
    if (prod == 1 && E.jp < 0) {
        // no slab above any more: jm loses its upper coupling
        float* CupM = I.Cup + Sm.offCup;
        if (chunk == 0)
            for (int t = tid; t < Sm.nm * Sm.ldc; t += nt) CupM[t] = 0.f;
        return;
    }
    // this CTA's rows [r0, r0 + M) of the product's M_all rows
    const int Mall = up ? Sm.nm : Sp.nv;
    const int mw = (Mall + nch - 1) / nch;
    const int r0 = min(Mall, chunk * mw);
    const int M = min(Mall, r0 + mw) - r0;
    if (M <= 0) return;
    const float* Lrows = (up ? Rup : Rdn) + (size_t)r0 * Sj.n;
    const int Mp = (M + 3) & ~3, Np = (N + 3) & ~3;
    float* Asm = esm;                   // (L Q)^T, Np x Mp
    float* stL = Asm + Np * Mp;         // 32 x (Mp + 4)
    float* stQ = stL + 32 * (Mp + 4);   // 32 x (Np + 4)
    float* Csm = stQ + 32 * (Np + 4);   // Np x (column chunk rounded up to 4)
    __syncthreads();
    rows_times_cols(Lrows, M, Sj.n, Dinv, np, cols, N, Asm, stL, stQ);
    if (prod == 0) {
        apply_coupling<true>(Asm, M, N, Cdn_j, Sj.ldc, Sm.n, Csm, I.elim_cw, I.D + Sm.offD, np,
                             I.idx + Sm.offIdx + r0, nullptr, 0, 0);
    } else if (prod == 1) {
        apply_coupling<false>(Asm, M, N, Cup_j, Sj.ldc, Sp.n, Csm, I.elim_cw, nullptr, np, nullptr,
                              I.Cup + Sm.offCup + (size_t)r0 * Sm.ldc, Sm.ldc, Sm.ldc);
    } else if (prod == 2) {
        apply_coupling<true>(Asm, M, N, Cup_j, Sj.ldc, Sp.n, Csm, I.elim_cw, I.D + Sp.offD, np,
                             I.idx + Sp.offIdx + Sp.nm + r0, nullptr, 0, 0);
    } else {
        apply_coupling<false>(Asm, M, N, Cdn_j, Sj.ldc, Sm.n, Csm, I.elim_cw, nullptr, np, nullptr,
                              I.Cdn + Sp.offCdn + (size_t)r0 * Sp.ldc, Sp.ldc, Sp.ldc);
    }
}

// ---------------------------------------------------------------------------
// Solve phase (per refinement step).
// ---------------------------------------------------------------------------
__global__ void k_if_residual(IfPtrs I, const int* row_member, int nrows, int first) {
    pdl_wait_and_release();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    const double* gv = I.Gv + (size_t)row * 2 * I.NB;
    double s = I.rhs[row];
    for (int b = 0; b < 2; ++b) {
        int c0 = I.Gc[2 * row + b], nc = I.Gn[2 * row + b];
        for (int k = 0; k < nc; ++k) s -= gv[b * I.NB + k] * I.x[c0 + k];
    }
    I.r[row] = s;
    const double rs = I.R[row] * s;
    I.bq[row] = (float)rs;
    // norms of the row-equilibrated residual and right-hand side: each row on
    // its own scale (the flux rows scale with K, the pressure rows do not)
    const int m = row_member[row];
    atomic_max_pos(&I.rnorm[2 * m], fabs(rs));
    if (first) atomic_max_pos(&I.rnorm[2 * m + 1], fabs(I.R[row] * I.rhs[row]));
}

// Warp-cooperative dot product of a row-major matrix row with a shared vector.
__device__ __forceinline__ float warp_dot(const float* row, const float* v, int n) {
    const int lane = threadIdx.x & 31;
    float acc = 0.f;
    for (int c = lane; c < n; c += 32) acc += row[c] * v[c];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// The sweeps of the reduction: one cluster of SW_CL CTAs per slab, so that
// the products with the slab inverse (n x n FP32, read from L2 / HBM) have
// SW_CL times the loads in flight of a single CTA.  Partial products over
// column chunks are summed through distributed shared memory in a fixed
// order (the result does not depend on timing).
constexpr int SW_CL = 8;
constexpr int SW_T = 256;

// forward: y_j = Dinv_j b_j (stored in place), then push into the neighbours:
// b_jm[mrows] -= Rup y_j, b_jp[vrows] -= Rdn y_j.
__global__ void __launch_bounds__(SW_T) k_bcr_fwd(IfPtrs I, const ElimDev* el, int nel) {
    pdl_wait_and_release();
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int e = blockIdx.x / SW_CL;   // the grid is nel clusters
    extern __shared__ __align__(16) float fsm[];
    const int np = I.npad;
    float* part = fsm;        // np: Dinv_j b_j over this CTA's column chunk
    float* y = fsm + np;      // np: y_j
    float* bs = y + np;       // the column chunk of b_j
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, nwarp = nt >> 5;
    const ElimDev E = el[e];
    const SlabDev Sj = I.slabs[E.j];
    const int n = Sj.n;
    const int cw = (n + SW_CL - 1) / SW_CL, c0 = min(n, rank * cw), c1 = min(n, c0 + cw);
    const float* Dinv = I.Dinv + Sj.offD;
    float* bj = I.bq + Sj.col0;
    for (int c = c0 + tid; c < c1; c += nt) bs[c - c0] = bj[c];
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int c = c0;
        for (; c + 3 < c1; c += 4) {
            a0 += Dinv[(size_t)c * np + r] * bs[c - c0];
            a1 += Dinv[(size_t)(c + 1) * np + r] * bs[c + 1 - c0];
            a2 += Dinv[(size_t)(c + 2) * np + r] * bs[c + 2 - c0];
            a3 += Dinv[(size_t)(c + 3) * np + r] * bs[c + 3 - c0];
        }
        for (; c < c1; ++c) a0 += Dinv[(size_t)c * np + r] * bs[c - c0];
        part[r] = (a0 + a1) + (a2 + a3);
    }
    cluster.sync();   // partials complete; every chunk of b_j read before it is overwritten
    for (int r = tid; r < n; r += nt) {
        float acc = 0.f;
        for (int q = 0; q < SW_CL; ++q) acc += cluster.map_shared_rank(part, q)[r];
        y[r] = acc;
    }
    cluster.sync();   // no CTA leaves while its partials may still be read
    if (rank == 0)
        for (int r = tid; r < n; r += nt) bj[r] = y[r];
    if (E.jm >= 0 && E.jm != E.j) {
        const SlabDev Sm = I.slabs[E.jm];
        const float* Rup = I.Rup + Sj.offRup;
        const int* mrows_m = I.idx + Sm.offIdx;
        float* bm = I.bq + Sm.col0;
        for (int r = rank * nwarp + warp; r < Sm.nm; r += SW_CL * nwarp) {
            const float acc = warp_dot(Rup + (size_t)r * n, y, n);
            if ((tid & 31) == 0) bm[mrows_m[r]] -= acc;
        }
    }
    if (E.jp >= 0) {
        const SlabDev Sp = I.slabs[E.jp];
        const float* Rdn = I.Rdn + Sj.offRdn;
        const int* vrows_p = I.idx + Sp.offIdx + Sp.nm;
        float* bp = I.bq + Sp.col0;
        for (int r = rank * nwarp + warp; r < Sp.nv; r += SW_CL * nwarp) {
            const float acc = warp_dot(Rdn + (size_t)r * n, y, n);
            if ((tid & 31) == 0) bp[vrows_p[r]] -= acc;
        }
    }
}

// backward: x_j = y_j - Dinv_j[:, vrows] (Cdn_j x_jm) - Dinv_j[:, mrows] (Cup_j x_jp).
// The coupling products are split over the cluster by rows (contiguous
// chunks, gathered through distributed shared memory), the products with
// the inverse columns by chunks of those columns, the final sum by rows.
__global__ void __launch_bounds__(SW_T) k_bcr_bwd(IfPtrs I, const ElimDev* el, int nel) {
    pdl_wait_and_release();
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int e = blockIdx.x / SW_CL;
    extern __shared__ __align__(16) float bsm[];
    const int np = I.npad;
    float* xm = bsm;              // n_jm
    float* xp = bsm + np;         // n_jp
    float* tl = bsm + 2 * np;     // this CTA's entries of (tv, tm), at their own positions
    float* tv = bsm + 3 * np;     // nv_j
    float* tm = bsm + 4 * np;     // nm_j
    float* part = bsm + 5 * np;   // np
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, nwarp = nt >> 5;
    const ElimDev E = el[e];
    const SlabDev Sj = I.slabs[E.j];
    const int n = Sj.n;
    const float* Dinv = I.Dinv + Sj.offD;
    const int* mrows_j = I.idx + Sj.offIdx;
    const int* vrows_j = mrows_j + Sj.nm;
    const SlabDev Sm = I.slabs[E.jm];
    for (int c = tid; c < Sm.n; c += nt) xm[c] = I.bq[Sm.col0 + c];
    const int nv = Sj.nv, nmj = E.jp >= 0 ? Sj.nm : 0, nq = nv + nmj;
    SlabDev Sp{};
    if (E.jp >= 0) {
        Sp = I.slabs[E.jp];
        for (int c = tid; c < Sp.n; c += nt) xp[c] = I.bq[Sp.col0 + c];
    }
    __syncthreads();
    // (tv, tm) entries q in [k0, k1) of the nq coupling rows (tv first)
    const int kw = (nq + SW_CL - 1) / SW_CL, k0 = min(nq, rank * kw), k1 = min(nq, k0 + kw);
    const float* Cdn_j = I.Cdn + Sj.offCdn;
    const float* Cup_j = I.Cup + Sj.offCup;
    for (int q = k0 + warp; q < k1; q += nwarp) {
        const float acc = q < nv ? warp_dot(Cdn_j + (size_t)q * Sj.ldc, xm, Sm.n)
                                 : warp_dot(Cup_j + (size_t)(q - nv) * Sj.ldc, xp, Sp.n);
        if ((tid & 31) == 0) tl[q] = acc;
    }
    cluster.sync();
    for (int q = tid; q < nq; q += nt) {
        const float v = cluster.map_shared_rank(tl, q / kw)[q];
        if (q < nv) tv[q] = v;
        else tm[q - nv] = v;
    }
    __syncthreads();
    // partial products over this CTA's chunk of the coupling columns
    for (int r = tid; r < n; r += nt) {
        float a0 = 0.f, a1 = 0.f;
        int q = k0;
        for (; q + 1 < k1; q += 2) {
            const int ca = q < nv ? vrows_j[q] : mrows_j[q - nv];
            const int cb = q + 1 < nv ? vrows_j[q + 1] : mrows_j[q + 1 - nv];
            a0 += Dinv[(size_t)ca * np + r] * (q < nv ? tv[q] : tm[q - nv]);
            a1 += Dinv[(size_t)cb * np + r] * (q + 1 < nv ? tv[q + 1] : tm[q + 1 - nv]);
        }
        if (q < k1) a0 += Dinv[(size_t)(q < nv ? vrows_j[q] : mrows_j[q - nv]) * np + r] * (q < nv ? tv[q] : tm[q - nv]);
        part[r] = a0 + a1;
    }
    cluster.sync();
    const int rw = (n + SW_CL - 1) / SW_CL, r0 = min(n, rank * rw), r1 = min(n, r0 + rw);
    float* xj = I.bq + Sj.col0;
    for (int r = r0 + tid; r < r1; r += nt) {
        float acc = 0.f;
        for (int q = 0; q < SW_CL; ++q) acc += cluster.map_shared_rank(part, q)[r];
        xj[r] -= acc;
    }
    cluster.sync();   // no CTA leaves while its shared memory may still be read
}

__global__ void k_if_update(IfPtrs I, int ncols) {
    pdl_wait_and_release();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    I.x[c] += I.Cs[c] * (double)I.bq[c];
}

// ---------------------------------------------------------------------------
// Transposed solve G^T y = z (the interface step of the adjoint).  The FP32
// block-cyclic-reduction factors of R G C are applied transposed:
//   (R G C)^-T = C^-1 ... : with M^-1 = B_0 ... B_{L-2} F_{L-1} ... F_0 the
// forward sweep (F_l per level, then B_l back down), M^-T applies B_l^T for
// l = 0 .. L-2 and then F_l^T for l = L-1 .. 0.  FP64 residuals of the
// unscaled G^T drive the refinement as in the forward solve:
//   r = z - G^T y,  bq = C r,  bq <- M^-T bq,  y += R bq.
// ---------------------------------------------------------------------------

// r = z - G^T y, gathered per column: the rows that reference column c are
// the owner's own rows (first block) and its neighbours' rows whose second
// block is the owner.
__global__ void k_if_residualT(IfPtrs I, const SubDev* sub, const int* col_item, const double* z,
                               const double* y, const int* row_member, int ncols, int first) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const SubDev sd = sub[col_item[c]];
    const int k = c - sd.col0;
    const int NB = I.NB;
    double s = z[c];
    for (int q = 0; q < sd.nbasis; ++q) {
        const int row = sd.col0 + q;
        s -= I.Gv[(size_t)row * 2 * NB + k] * y[row];
    }
    for (int sid = 0; sid < MRCM_MAXSIDE; ++sid) {
        const int t = sd.nbr[sid];
        if (t < 0) continue;
        const SubDev st = sub[t];
        for (int q = 0; q < st.nbasis; ++q) {
            const int row = st.col0 + q;
            if (I.Gc[2 * row + 1] == sd.col0) s -= I.Gv[(size_t)row * 2 * NB + NB + k] * y[row];
        }
    }
    I.r[c] = s;
    const double cs = I.Cs[c] * s;
    I.bq[c] = (float)cs;
    const int m = row_member[c];
    atomic_max_pos(&I.rnorm[2 * m], fabs(cs));
    if (first) atomic_max_pos(&I.rnorm[2 * m + 1], fabs(I.Cs[c] * z[c]));
}

// B_l^T for the eliminations of one level: v_jm -= Cdn_j^T (Dinv_j[:, vrows]^T v_j)
// (up = 0) or v_jp -= Cup_j^T (Dinv_j[:, mrows]^T v_j) (up = 1).  Each
// surviving slab receives from one elimination per launch.
__global__ void __launch_bounds__(SW_T) k_bcr_bwdT(IfPtrs I, const ElimDev* el, int nel, int up) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int e = blockIdx.x / SW_CL;   // the grid is nel clusters
    extern __shared__ __align__(16) float tsm[];
    const ElimDev E = el[e];
    if (up && E.jp < 0) return;   // uniform over the cluster
    const SlabDev Sj = I.slabs[E.j];
    const int np = I.npad;
    const float* Dinv = I.Dinv + Sj.offD;
    const int* rows = I.idx + Sj.offIdx + (up ? 0 : Sj.nm);
    const int nq = up ? Sj.nm : Sj.nv;
    float* vj = tsm;           // n_j
    float* tl = tsm + np;      // this CTA's entries of t, at their own positions
    float* t = tsm + 2 * np;   // nq
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, nwarp = nt >> 5;
    for (int r = tid; r < Sj.n; r += nt) vj[r] = I.bq[Sj.col0 + r];
    __syncthreads();
    // t = Dinv_j[:, rows]^T v_j, the entries split over the cluster in contiguous chunks
    const int kw = (nq + SW_CL - 1) / SW_CL, k0 = min(nq, rank * kw), k1 = min(nq, k0 + kw);
    for (int q = k0 + warp; q < k1; q += nwarp) {
        const float acc = warp_dot(Dinv + (size_t)rows[q] * np, vj, Sj.n);
        if ((tid & 31) == 0) tl[q] = acc;
    }
    cluster.sync();
    for (int q = tid; q < nq; q += nt) t[q] = cluster.map_shared_rank(tl, q / kw)[q];
    cluster.sync();   // no CTA leaves while its entries may still be read
    // b_t -= C^T t over this CTA's chunk of the target entries
    const SlabDev St = I.slabs[up ? E.jp : E.jm];
    const float* Cq = I.Cup + (up ? Sj.offCup : Sj.offCdn);
    float* bt = I.bq + St.col0;
    const int cwd = (St.n + SW_CL - 1) / SW_CL, c0 = min(St.n, rank * cwd), c1 = min(St.n, c0 + cwd);
    for (int c = c0 + tid; c < c1; c += nt) {
        float acc = 0.f;
        for (int q = 0; q < nq; ++q) acc += Cq[(size_t)q * Sj.ldc + c] * t[q];
        bt[c] -= acc;
    }
}

// F_l^T for the eliminations of one level:
// b_j -= Rup^T b_jm[mrows_jm] + Rdn^T b_jp[vrows_jp], then b_j <- Dinv_j^T b_j.
__global__ void __launch_bounds__(SW_T) k_bcr_fwdT(IfPtrs I, const ElimDev* el, int nel) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int e = blockIdx.x / SW_CL;
    extern __shared__ __align__(16) float fts[];
    const ElimDev E = el[e];
    const SlabDev Sj = I.slabs[E.j];
    const int np = I.npad, n = Sj.n;
    float* part = fts;         // np: neighbour terms over this CTA's chunk of coupling rows
    float* bs = fts + np;      // np: b_j after the neighbour terms
    float* gv = fts + 2 * np;  // 2 np: the neighbours' coupled entries (m rows, then v rows)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, nwarp = nt >> 5;
    const bool hm = E.jm >= 0 && E.jm != E.j, hp = E.jp >= 0;
    SlabDev Sm{}, Sp{};
    int nmm = 0, nvp = 0;
    if (hm) {
        Sm = I.slabs[E.jm];
        nmm = Sm.nm;
        const int* mrows_m = I.idx + Sm.offIdx;
        for (int q = tid; q < nmm; q += nt) gv[q] = I.bq[Sm.col0 + mrows_m[q]];
    }
    if (hp) {
        Sp = I.slabs[E.jp];
        nvp = Sp.nv;
        const int* vrows_p = I.idx + Sp.offIdx + Sp.nm;
        for (int q = tid; q < nvp; q += nt) gv[nmm + q] = I.bq[Sp.col0 + vrows_p[q]];
    }
    __syncthreads();
    const float* Rup = I.Rup + Sj.offRup;   // nm_jm x n_j
    const float* Rdn = I.Rdn + Sj.offRdn;   // nv_jp x n_j
    const int nq = nmm + nvp;
    const int kw = (nq + SW_CL - 1) / SW_CL, k0 = min(nq, rank * kw), k1 = min(nq, k0 + kw);
    for (int r = tid; r < n; r += nt) {
        float acc = 0.f;
        for (int q = k0; q < k1; ++q)
            acc += (q < nmm ? Rup[(size_t)q * n + r] : Rdn[(size_t)(q - nmm) * n + r]) * gv[q];
        part[r] = acc;
    }
    cluster.sync();   // partials complete; every read of b_j below precedes the writes after the next barrier
    for (int r = tid; r < n; r += nt) {
        float acc = 0.f;
        for (int q = 0; q < SW_CL; ++q) acc += cluster.map_shared_rank(part, q)[r];
        bs[r] = I.bq[Sj.col0 + r] - acc;
    }
    cluster.sync();   // no CTA leaves while its partials may still be read, b_j read by all
    // b_j <- Dinv_j^T b_j, the rows split over the cluster
    const float* Dinv = I.Dinv + Sj.offD;
    const int rw = (n + SW_CL - 1) / SW_CL, r0 = min(n, rank * rw), r1 = min(n, r0 + rw);
    for (int r = r0 + warp; r < r1; r += nwarp) {
        const float acc = warp_dot(Dinv + (size_t)r * np, bs, n);
        if ((tid & 31) == 0) I.bq[Sj.col0 + r] = acc;
    }
}

__global__ void k_if_updateT(IfPtrs I, double* y, int nrows) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    y[r] += I.R[r] * (double)I.bq[r];
}

cudaError_t if_residualT(const IfPtrs& I, const SubDev* sub, const int* col_item, const double* z,
                         const double* y, const int* row_member, int n, int first, cudaStream_t s) {
    k_if_residualT<<<(n + 255) / 256, 256, 0, s>>>(I, sub, col_item, z, y, row_member, n, first);
    return cudaGetLastError();
}

static cudaError_t launch_cluster(const void* kern, int nblocks, int threads, size_t smem, cudaStream_t s,
                                  void** args, int cl = GJ_CL, bool pdl = false) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelExC(&cfg, kern, args);
}

cudaError_t bcr_bwdT(const IfPtrs& I, const ElimDev* el, int nel, int nmax, int up, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel, &up};
    return launch_cluster((const void*)k_bcr_bwdT, nel * SW_CL, SW_T, sizeof(float) * 3 * (size_t)nmax, s, args, SW_CL);
}

cudaError_t bcr_fwdT(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel};
    return launch_cluster((const void*)k_bcr_fwdT, nel * SW_CL, SW_T, sizeof(float) * 4 * (size_t)nmax, s, args, SW_CL);
}

cudaError_t if_updateT(const IfPtrs& I, double* y, int n, cudaStream_t s) {
    k_if_updateT<<<(n + 255) / 256, 256, 0, s>>>(I, y, n);
    return cudaGetLastError();
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


cudaError_t if_residual(const IfPtrs& I, const int* row_member, int nrows, int first, cudaStream_t s) {
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&row_member, &nrows, &first};
    return launch_cluster((const void*)k_if_residual, (nrows + 255) / 256, 256, 0, s, args, 1, true);
}

cudaError_t bcr_fwd(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel};
    const size_t smem = sizeof(float) * (2 * (size_t)nmax + (nmax + SW_CL - 1) / SW_CL);
    return launch_cluster((const void*)k_bcr_fwd, nel * SW_CL, SW_T, smem, s, args, SW_CL, true);
}

cudaError_t bcr_bwd(const IfPtrs& I, const ElimDev* el, int nel, int nmax, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel};
    const size_t smem = sizeof(float) * 6 * (size_t)nmax;
    return launch_cluster((const void*)k_bcr_bwd, nel * SW_CL, SW_T, smem, s, args, SW_CL, true);
}

cudaError_t if_update(const IfPtrs& I, int ncols, cudaStream_t s) {
    IfPtrs Ic = I;
    void* args[] = {&Ic, &ncols};
    return launch_cluster((const void*)k_if_update, (ncols + 255) / 256, 256, 0, s, args, 1, true);
}

// ---------------------------------------------------------------------------
// Slab inverse through a blocked LU factorisation with partial pivoting
// (FP32, column-major np x np, in place in D, inverse written to Dinv).
// X <- L11^-1 X (LOWER, unit diagonal) or U11^-1 X on the rows of one
// diagonal block by substitution, for nb right-hand sides: T holds the
// factored block (T[c2 * ldt + c] = entry (c, c2), b x b, b a multiple of 4),
// the entry (c, jj) of X is X[c * rs + jj * cs].  Eight consecutive lanes
// share a right-hand side, four rows each; the entry solved at each step is
// passed within the eight by a shuffle, so no barrier is needed and every
// thread reads and writes only its own rows (up to four passes of the block
// for nb <= 256).  The diagonal of U is applied as a correctly rounded
// reciprocal; a zero pivot (already flagged singular) is taken as 1e-30.
template <bool LOWER>
__device__ void diag_solve(const float* __restrict__ T, int ldt, float* X, int rs, int cs, int b, int nb) {
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        const int w = threadIdx.x + k * blockDim.x;
        if (w - lane >= 8 * nb) break;   // warp-uniform: the whole warp is past the last right-hand side
        const bool own = w < 8 * nb;
        const int g = w & 7, jj = w >> 3;
        float x[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = (own && 4 * g + e < b) ? X[(4 * g + e) * rs + jj * cs] : 0.f;
        if (LOWER) {
#pragma unroll
            for (int c = 0; c < GJ_NB; ++c) {
                if (c < b) {
                    const float xc = __shfl_sync(0xffffffffu, x[c & 3], c >> 2, 8);
                    const float4 t = *reinterpret_cast<const float4*>(T + c * ldt + 4 * g);
                    if (4 * g + 0 > c) x[0] -= t.x * xc;
                    if (4 * g + 1 > c) x[1] -= t.y * xc;
                    if (4 * g + 2 > c) x[2] -= t.z * xc;
                    if (4 * g + 3 > c) x[3] -= t.w * xc;
                }
            }
        } else {
#pragma unroll
            for (int c = GJ_NB - 1; c >= 0; --c) {
                if (c < b) {
                    float d = T[c * ldt + c];
                    if (d == 0.f) d = 1e-30f;
                    if (g == (c >> 2)) x[c & 3] *= __frcp_rn(d);
                    const float xc = __shfl_sync(0xffffffffu, x[c & 3], c >> 2, 8);
                    const float4 t = *reinterpret_cast<const float4*>(T + c * ldt + 4 * g);
                    if (4 * g + 0 < c) x[0] -= t.x * xc;
                    if (4 * g + 1 < c) x[1] -= t.y * xc;
                    if (4 * g + 2 < c) x[2] -= t.z * xc;
                    if (4 * g + 3 < c) x[3] -= t.w * xc;
                }
            }
        }
        if (own) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (4 * g + e < b) X[(4 * g + e) * rs + jj * cs] = x[e];
        }
    }
}

// Phase 1 (cluster-synchronised per panel of GJ_NB columns): every CTA of
// the cluster factors the panel redundantly in shared memory and inverts its
// unit-lower and upper diagonal blocks; the owner writes the panel and the
// two block inverses back, and each CTA applies the interchanges to the
// columns it owns, forms their U12 rows (L11^-1 A12) and updates their
// trailing part (A22 -= L21 U12).
// Phase 2 (independent per CTA): the columns of the inverse owned by a CTA
// are solved from P A = L U (column j = U^-1 L^-1 e_{q(j)}) panel by panel,
// each diagonal block applied through its kept inverse.
// ---------------------------------------------------------------------------

// X[r][jj] -= sum_c P[r][c] X[k0 + c][jj] for rows r in [ra, rb) and the
// first nb columns of X (column-major, ld np), with P the panel (column-major,
// ld np) -- 4 x 4 register tiles (ra, rb, nb multiples of 4).
__device__ void tile_update(const float* __restrict__ P, float* __restrict__ X, int np, int k0, int b, int ra,
                            int rb, int nb) {
    const int ntr = (rb - ra) >> 2, ntc = nb >> 2;
    for (int t = threadIdx.x; t < ntr * ntc; t += blockDim.x) {
        const int tc = t / ntr;
        const int r = ra + ((t - tc * ntr) << 2), jj0 = tc << 2;
        float acc[4][4];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const float4 v = *reinterpret_cast<const float4*>(&X[(jj0 + y) * np + r]);
            acc[0][y] = v.x; acc[1][y] = v.y; acc[2][y] = v.z; acc[3][y] = v.w;
        }
        for (int c = 0; c < b; ++c) {
            const float4 s4 = *reinterpret_cast<const float4*>(&P[c * np + r]);
            const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
            float xv[4];
#pragma unroll
            for (int y = 0; y < 4; ++y) xv[y] = X[(jj0 + y) * np + k0 + c];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] -= sv[x] * xv[y];
        }
#pragma unroll
        for (int y = 0; y < 4; ++y)
            *reinterpret_cast<float4*>(&X[(jj0 + y) * np + r]) = make_float4(acc[0][y], acc[1][y], acc[2][y], acc[3][y]);
    }
}

template <int RPT>
__global__ void __launch_bounds__(GJ_THREADS) k_lu_inverse(IfPtrs I, const ElimDev* el, int nel, int* status) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int e = blockIdx.x / CL;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
    const int np = I.npad;
    const int npan = (np + GJ_NB - 1) / GJ_NB;
    const int ncmax = ((npan + CL - 1) / CL) * GJ_NB;
    extern __shared__ __align__(16) float lsm[];
    float* Ps = lsm;                           // [c][r], GJ_NB * np
    float* Xs = Ps + GJ_NB * np;                          // phase 1 [c][jj] (ld ncmax), phase 2 [jj][r]
    const int XCH = I.xch;
    float* Upy = Xs + max(GJ_NB * ncmax, XCH * np);       // [c][jj], max(GJ_NB * ncmax, np)
    int* piv = (int*)(Upy + max(GJ_NB * ncmax, np));  // np
    int* ownc = piv + np;                      // ncmax
    int* qpos = ownc + ncmax;                  // np
    float* pub = reinterpret_cast<float*>(qpos + np);   // 2 x PUB_PAR candidate rows published per column
    unsigned* pkey = reinterpret_cast<unsigned*>(pub + PUB_FLOATS);   // 2 x GJ_NB_WARPS pivot keys
    int* rowperm = reinterpret_cast<int*>(pkey + 2 * GJ_NB_WARPS);    // np: original row at each position
    __shared__ int nown;
    __shared__ int aff[2 * GJ_NB];
    __shared__ int naff;
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
        for (int q = rank; q < npan; q += CL)
            for (int j = q * GJ_NB; j < min(np, (q + 1) * GJ_NB); ++j) ownc[c++] = j;
        nown = c;
    }
    for (int i = tid; i < np; i += nt) rowperm[i] = i;
    bool singular = false;
    // ---------------- phase 1: P A = L U ----------------
    for (int q = 0; q < npan; ++q) {
        __threadfence();
        cluster.sync();
        const int k0 = q * GJ_NB, b = min(GJ_NB, np - k0);
        if (active)
            for (int c = warp; c < b; c += nwarp)
                for (int r = k0 + lane; r < np; r += 32) Ps[c * np + r] = __ldcg(&A[(size_t)(k0 + c) * np + r]);
        cluster.sync();
        if (!active) continue;
        // panel factorisation with partial pivoting.  Every thread keeps its
        // RPT panel rows (slots k0 + tid + 512 i) in registers for the whole
        // panel and never moves them; it tracks the logical row each slot
        // holds, so a row interchange is two integer updates.  The registers
        // rotate left after every column, so the pivot column is always x[0]
        // and the column loop stays one short body.  One barrier per column:
        // before it each warp reduces its pivot candidate by one redux and
        // publishes that row; after it every warp picks the winner among the
        // warps' keys by one more.  A key is |a| with its 11 low mantissa
        // bits replaced by 2047 - (logical row - r0): the largest magnitude
        // to 2^-12 relative wins, the first row among equals (threshold
        // partial pivoting).  The published rows are double-buffered by the
        // column's parity.  Each step leaves column c of every slot in Ps;
        // the slots are put into logical row order once the panel is done.
        {
            float x[RPT][GJ_NB];
            int lp[RPT];
            const bool wact = k0 + warp * 32 < np;   // the warp holds at least one panel row
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int r = k0 + tid + i * nt;
                lp[i] = r;
#pragma unroll
                for (int cc = 0; cc < GJ_NB; ++cc) x[i][cc] = (r < np && cc < b) ? Ps[cc * np + r] : 0.f;
            }
#pragma unroll 1
            for (int c = 0; c < b; ++c) {
                const int r0 = k0 + c, par = c & 1;
                float* pb = pub + par * PUB_PAR;            // [warp][GJ_NB] candidate rows
                if (!wact) {
                    // a warp without panel rows only takes part in the column's barrier
                    if (lane == 0) pkey[par * GJ_NB_WARPS + warp] = 0u;
                    __syncthreads();
                    continue;
                }
                unsigned key = 0u;   // 0: no candidate; a candidate's key is at least 1024 (np <= 1024)
                int ks = -1;
#pragma unroll
                for (int i = 0; i < RPT; ++i) {
                    if (lp[i] >= r0 && lp[i] < np) {
                        const float v = fabsf(x[i][0]);
                        const unsigned kb = ((v == v ? __float_as_uint(v) : 0u) & ~0x7ffu) | (0x7ffu - (unsigned)(lp[i] - r0));
                        if (kb > key) { key = kb; ks = i; }
                    }
                }
                const unsigned m = __reduce_max_sync(0xffffffffu, key);
#pragma unroll
                for (int i = 0; i < RPT; ++i)
                    if (ks == i && key == m) {
                        float4* dst = reinterpret_cast<float4*>(pb + warp * GJ_NB);
#pragma unroll
                        for (int q4 = 0; q4 < GJ_NB / 4; ++q4)
                            dst[q4] = make_float4(x[i][4 * q4], x[i][4 * q4 + 1], x[i][4 * q4 + 2], x[i][4 * q4 + 3]);
                    }
                if (lane == 0) pkey[par * GJ_NB_WARPS + warp] = m;
                __syncthreads();
                const unsigned km = lane < GJ_NB_WARPS ? pkey[par * GJ_NB_WARPS + lane] : 0u;
                const unsigned bm = __reduce_max_sync(0xffffffffu, km);
                const unsigned p = (unsigned)r0 + 0x7ffu - (bm & 0x7ffu);
                const unsigned wb = __ballot_sync(0xffffffffu, km == bm && bm != 0u);
                if (wb == 0u) {
                    // no candidate anywhere (cannot happen while r0 < np): keep the order, flag it
                    singular = true;
                    if (tid == 0) piv[r0] = r0;
                } else {
                    const int pw = __ffs(wb) - 1;
                    if (tid == 0) piv[r0] = (int)p;
                    const float4* src = reinterpret_cast<const float4*>(pb + pw * GJ_NB);
                    float a = pb[pw * GJ_NB];
                    if (a == 0.f) { singular = true; a = 1e-30f; }
                    const float ia = __frcp_rn(a);   // correctly rounded, equal to 1.f / a
#pragma unroll
                    for (int i = 0; i < RPT; ++i) {
                        if ((unsigned)lp[i] == p) lp[i] = r0;
                        else if (lp[i] == r0) lp[i] = (int)p;
                        if (lp[i] > r0 && lp[i] < np) {
                            const float l = x[i][0] * ia;
                            x[i][0] = l;
#pragma unroll
                            for (int q4 = 0; q4 < GJ_NB / 4; ++q4) {
                                const float4 t = src[q4];
                                if (q4 > 0) x[i][4 * q4] -= l * t.x;
                                x[i][4 * q4 + 1] -= l * t.y;
                                x[i][4 * q4 + 2] -= l * t.z;
                                x[i][4 * q4 + 3] -= l * t.w;
                            }
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < RPT; ++i) {
                    const int sl = k0 + tid + i * nt;
                    if (sl < np) Ps[c * np + sl] = x[i][0];
#pragma unroll
                    for (int cc = 0; cc < GJ_NB - 1; ++cc) x[i][cc] = x[i][cc + 1];
                    x[i][GJ_NB - 1] = 0.f;
                }
            }
            // slots into logical row order
            __syncthreads();
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int sl = k0 + tid + i * nt;
#pragma unroll
                for (int cc = 0; cc < GJ_NB; ++cc) x[i][cc] = (sl < np && cc < b) ? Ps[cc * np + sl] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                if (k0 + tid + i * nt < np) {
#pragma unroll
                    for (int cc = 0; cc < GJ_NB; ++cc)
                        if (cc < b) Ps[cc * np + lp[i]] = x[i][cc];
                }
            }
        }
        __syncthreads();
        // interchanges on owned columns: the panel's swaps composed into one
        // permutation of at most 2 GJ_NB rows, then gathered column by column
        for (int i = k0 + tid; i < np; i += nt) qpos[i] = i;
        __syncthreads();
        if (tid == 0) {
            for (int c = 0; c < b; ++c) {
                const int p = piv[k0 + c], t0 = qpos[k0 + c];
                qpos[k0 + c] = qpos[p];
                qpos[p] = t0;
            }
            naff = 0;
        }
        __syncthreads();
        for (int i = k0 + tid; i < np; i += nt)
            if (qpos[i] != i) aff[atomicAdd(&naff, 1)] = i;
        __syncthreads();
        {
            // the panel's interchanges applied to the row permutation
            const int na = naff;
            const int rv = tid < na ? rowperm[qpos[aff[tid]]] : 0;
            __syncthreads();
            if (tid < na) rowperm[aff[tid]] = rv;
        }
        const int no = nown;
        for (int jj = warp; jj < no; jj += nwarp) {
            const int j = ownc[jj];
            if (j >= k0 && j < k0 + b) continue;
            float* col = A + (size_t)j * np;
            float v0 = 0.f, v1 = 0.f;
            if (lane < naff) v0 = col[qpos[aff[lane]]];
            if (lane + 32 < naff) v1 = col[qpos[aff[lane + 32]]];
            __syncwarp();
            if (lane < naff) col[aff[lane]] = v0;
            if (lane + 32 < naff) col[aff[lane + 32]] = v1;
        }
        __syncthreads();
        if (q % CL == rank)
            for (int c = warp; c < b; c += nwarp)
                for (int r = k0 + lane; r < np; r += 32) A[(size_t)(k0 + c) * np + r] = Ps[c * np + r];
        // U12 = L11^-1 A12 on owned trailing columns (zero on the others): the
        // block rows staged in Upy, solved with the unit L11, written back
        for (int w = tid; w < GJ_NB * no; w += nt) {
            const int jj = w % no, c = w / no, j = ownc[jj];
            Upy[c * ncmax + jj] = (j >= k0 + b && c < b) ? A[(size_t)j * np + k0 + c] : 0.f;
        }
        __syncthreads();
        diag_solve<true>(Ps + k0, np, Upy, ncmax, 1, b, no);
        __syncthreads();
        for (int w = tid; w < b * no; w += nt) {
            const int jj = w % no, c = w / no, j = ownc[jj];
            if (j >= k0 + b) A[(size_t)j * np + k0 + c] = Upy[c * ncmax + jj];
        }
        // trailing update A22 -= L21 U12 over owned trailing columns
        const int r1 = k0 + b;
        if (r1 < np) {
            const int ntr = (np - r1) / 4, ntc = (no + 3) / 4;
            for (int t = tid; t < ntr * ntc; t += nt) {
                const int tc = t / ntr;
                const int r = r1 + (t - tc * ntr) * 4, jj0 = tc * 4;
                float acc[4][4];
                int jcol[4];
                bool skip[4];
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int jj = jj0 + y;
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
                    for (int y = 0; y < 4; ++y) av[y] = (jj0 + y < no) ? Upy[c * ncmax + jj0 + y] : 0.f;
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
    for (int i = tid; i < np; i += nt) qpos[rowperm[i]] = i;   // the inverse permutation
    __syncthreads();
    const int no = nown;
    for (int j0 = 0; j0 < no; j0 += XCH) {
        const int nb = min(XCH, no - j0);
        for (int jj = warp; jj < XCH; jj += nwarp)
            for (int r = lane; r < np; r += 32) Xs[jj * np + r] = (jj < nb && r == qpos[ownc[j0 + jj]]) ? 1.f : 0.f;
        __syncthreads();
        // forward with unit L
        for (int q = 0; q < npan; ++q) {
            const int k0 = q * GJ_NB, b = min(GJ_NB, np - k0);
            for (int c = warp; c < b; c += nwarp)
                for (int r = k0 + lane; r < np; r += 32) Ps[c * np + r] = __ldcg(&A[(size_t)(k0 + c) * np + r]);
            __syncthreads();
            diag_solve<true>(Ps + k0, np, Xs + k0, 1, np, b, nb);
            __syncthreads();
            tile_update(Ps, Xs, np, k0, b, k0 + b, np, nb);
            __syncthreads();
        }
        // backward with U
        for (int q = npan - 1; q >= 0; --q) {
            const int k0 = q * GJ_NB, b = min(GJ_NB, np - k0);
            for (int c = warp; c < b; c += nwarp)
                for (int r = lane; r < k0; r += 32) Ps[c * np + r] = __ldcg(&A[(size_t)(k0 + c) * np + r]);
            for (int c = warp; c < b; c += nwarp)
                for (int r = k0 + lane; r < k0 + b; r += 32) Ps[c * np + r] = __ldcg(&A[(size_t)(k0 + c) * np + r]);
            __syncthreads();
            diag_solve<false>(Ps + k0, np, Xs + k0, 1, np, b, nb);
            __syncthreads();
            tile_update(Ps, Xs, np, k0, b, 0, k0, nb);
            __syncthreads();
        }
        for (int jj = warp; jj < nb; jj += nwarp)
            for (int r = lane; r < np; r += 32) Ainv[(size_t)ownc[j0 + jj] * np + r] = Xs[jj * np + r];
        __syncthreads();
    }
    if (singular && tid == 0) atomicOr(status, ST_SINGULAR);
}

// ---------------------------------------------------------------------------
// Slab inverse by blocked Gauss-Jordan elimination with partial pivoting
// (FP32, in place) for slabs of at most GJI_T unknowns.  One cluster of CL
// CTAs per slab; CTA r owns the panels q = r, r + CL, ... of GJI_NB columns in
// shared memory.  For panel q its owner eliminates the panel's columns from
// ALL rows (Gauss-Jordan), choosing each pivot among the rows not yet used as
// pivots with the threshold rule of the slab LU (largest magnitude to 2^-12
// relative, first row among equals); the panel then holds its transformed
// columns P.  Every CTA applies the panel's row interchanges to its other
// columns and adds (P - E_K) A[K, J], K the panel's pivot rows: a rank-NB
// update.  After the last panel the storage holds (P_r A)^-1 for the
// accumulated row permutation P_r, and column i goes to column rowperm[i] of
// the inverse (A^-1 = (P_r A)^-1 P_r).  n^3 flops in one pass, against 2 n^3
// for the LU factors followed by the inverse columns.
// ---------------------------------------------------------------------------
constexpr int GJI_T = 256;                 // threads per CTA: one panel row each
constexpr int GJI_W = GJI_T / 32;
constexpr int GJI_NB = 8;                  // panel width (the composite update of wider panels loses accuracy)

size_t gji_smem(int np, int cl) {
    const int npan = (np + GJI_NB - 1) / GJI_NB;
    const int nq = (npan + cl - 1) / cl;   // panels owned by one CTA at most
    return sizeof(float) * ((size_t)nq * GJI_NB * np + (size_t)GJI_NB * np + (size_t)GJI_NB * nq * GJI_NB +
                            2 * GJI_W * GJI_NB) +
           sizeof(int) * ((size_t)2 * np + 4 * GJI_NB + 2 * GJI_W) + 64;
}

__global__ void __launch_bounds__(GJI_T) k_gj_inverse(IfPtrs I, const ElimDev* el, int nel, int* status) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int e = blockIdx.x / CL;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int np = I.npad;
    const int npan = (np + GJI_NB - 1) / GJI_NB;
    const int nqmax = (npan + CL - 1) / CL;
    const int nq = rank < npan ? (npan - rank + CL - 1) / CL : 0;   // panels this CTA owns
    const int ncol = nq * GJI_NB;                                  // owned column slots
    extern __shared__ __align__(16) float gsm[];
    float* Aown = gsm;                                       // [slot][np]: slot = local panel * NB + c
    float* Pt = Aown + (size_t)nqmax * GJI_NB * np;          // [c][np]: P - E_K of the current panel
    float* Tt = Pt + (size_t)GJI_NB * np;                    // [c][slot]: rows K of the owned columns
    float* pub = Tt + (size_t)GJI_NB * nqmax * GJI_NB;       // [2][warp][NB] published candidate rows
    int* rowperm = reinterpret_cast<int*>(pub + 2 * GJI_W * GJI_NB);   // [np] original row at each position
    int* qpos = rowperm + np;                                // [np]
    int* piv = qpos + np;                                    // [NB] the panel's pivot positions
    int* aff = piv + GJI_NB;                                 // [2 NB] rows moved by the panel's interchanges
    unsigned* pkey = reinterpret_cast<unsigned*>(aff + 2 * GJI_NB);    // [2][warp]
    __shared__ int naff;
    const bool active = e < nel;
    const float* A = nullptr;
    float* Ainv = nullptr;
    if (active) {
        const SlabDev S = I.slabs[el[e].j];
        A = I.D + S.offD;
        Ainv = I.Dinv + S.offD;
        for (int s = warp; s < ncol; s += GJI_W) {
            const int j = ((s / GJI_NB) * CL + rank) * GJI_NB + (s % GJI_NB);
            for (int r = lane; r < np; r += 32) Aown[(size_t)s * np + r] = j < np ? __ldcg(&A[(size_t)j * np + r]) : 0.f;
        }
    }
    for (int i = tid; i < np; i += nt) rowperm[i] = i;
    bool singular = false;
    __syncthreads();
    for (int q = 0; q < npan; ++q) {
        const int k0 = q * GJI_NB, b = min(GJI_NB, np - k0);
        const int owner = q % CL, ql = q / CL;               // owner and its local panel index
        const int par0 = 0;
        (void)par0;
        if (rank == owner && active) {
            // ---- the panel: rows in registers (slot tid), logical positions lp ----
            float x[GJI_NB];
            const bool row = tid < np;
            int lp = tid;
            const float* pcol = Aown + (size_t)ql * GJI_NB * np;
#pragma unroll
            for (int c = 0; c < GJI_NB; ++c) x[c] = (row && c < b) ? pcol[(size_t)c * np + tid] : 0.f;
#pragma unroll 1
            for (int c = 0; c < b; ++c) {
                const int r0 = k0 + c, par = c & 1;
                float* pb = pub + par * GJI_W * GJI_NB;
                unsigned key = 0u;
                if (row && lp >= r0) {
                    const float v = fabsf(x[0]);
                    key = ((v == v ? __float_as_uint(v) : 0u) & ~0x7ffu) | (0x7ffu - (unsigned)(lp - r0));
                }
                const unsigned m = __reduce_max_sync(0xffffffffu, key);
                if (key == m && m != 0u) {
                    float4* dst = reinterpret_cast<float4*>(pb + warp * GJI_NB);
#pragma unroll
                    for (int q4 = 0; q4 < GJI_NB / 4; ++q4)
                        dst[q4] = make_float4(x[4 * q4], x[4 * q4 + 1], x[4 * q4 + 2], x[4 * q4 + 3]);
                }
                if (lane == 0) pkey[par * GJI_W + warp] = m;
                __syncthreads();
                const unsigned km = lane < GJI_W ? pkey[par * GJI_W + lane] : 0u;
                const unsigned bm = __reduce_max_sync(0xffffffffu, km);
                const unsigned wb = __ballot_sync(0xffffffffu, km == bm && bm != 0u);
                if (wb == 0u) {
                    // no candidate (cannot happen while r0 < np): keep the order, flag it
                    singular = true;
                    if (tid == 0) piv[c] = r0;
                    // column c: nothing to eliminate; the rotation below keeps the column order
                } else {
                    const int pw = __ffs(wb) - 1;
                    const int p = r0 + 0x7ff - (int)(bm & 0x7ffu);
                    if (tid == 0) piv[c] = p;
                    const float4* src = reinterpret_cast<const float4*>(pb + pw * GJI_NB);
                    float a = pb[pw * GJI_NB];
                    if (a == 0.f) { singular = true; a = 1e-30f; }
                    const float ip = __frcp_rn(a);
                    if (lp == p) lp = r0;
                    else if (lp == r0) lp = p;
                    const bool isp = lp == r0;
                    // pivot row: ip * row; other rows: row - (a_rc ip) * pivot row; column c takes ip / -a_rc ip
                    const float f = x[0] * ip;
                    const float g = isp ? -ip : f;
                    const float c0 = isp ? ip : -f;
#pragma unroll
                    for (int q4 = 0; q4 < GJI_NB / 4; ++q4) {
                        const float4 t = src[q4];
                        if (q4 > 0) x[4 * q4] = (isp ? 0.f : x[4 * q4]) - g * t.x;
                        x[4 * q4 + 1] = (isp ? 0.f : x[4 * q4 + 1]) - g * t.y;
                        x[4 * q4 + 2] = (isp ? 0.f : x[4 * q4 + 2]) - g * t.z;
                        x[4 * q4 + 3] = (isp ? 0.f : x[4 * q4 + 3]) - g * t.w;
                    }
                    x[0] = c0;
                }
                // rotate left with wrap-around: the next pivot column is x[0]
                const float x0 = x[0];
#pragma unroll
                for (int cc = 0; cc < GJI_NB - 1; ++cc) x[cc] = x[cc + 1];
                x[GJI_NB - 1] = x0;
            }
            // after b rotations register rr holds column (rr + b) mod NB; write the panel in
            // logical row order, and P - E_K
            if (row) {
                float* dst = Aown + (size_t)ql * GJI_NB * np;
#pragma unroll
                for (int rr = 0; rr < GJI_NB; ++rr) {
                    int c = rr + b;
                    c = c >= GJI_NB ? c - GJI_NB : c;
                    if (c < b) {
                        dst[(size_t)c * np + lp] = x[rr];
                        Pt[(size_t)c * np + lp] = x[rr] - (lp == k0 + c ? 1.f : 0.f);
                    }
                }
            }
        }
        __threadfence();
        cluster.sync();   // the panel (P - E_K) and its pivots are in the owner's shared memory
        if (!active) continue;
        if (rank != owner) {
            const float* rP = cluster.map_shared_rank(Pt, owner);
            const int* rpiv = cluster.map_shared_rank(piv, owner);
            const float4* s4 = reinterpret_cast<const float4*>(rP);
            float4* d4 = reinterpret_cast<float4*>(Pt);
            for (int t = tid; t < (b * np) / 4; t += nt) d4[t] = s4[t];
            for (int t = (b * np) / 4 * 4 + tid; t < b * np; t += nt) Pt[t] = rP[t];
            if (tid < b) piv[tid] = rpiv[tid];
        }
        // the panel's interchanges composed into one permutation of at most 2 NB positions
        for (int i = tid; i < np; i += nt) qpos[i] = i;
        __syncthreads();
        if (tid == 0) {
            for (int c = 0; c < b; ++c) {
                const int p = piv[c], t0 = qpos[k0 + c];
                qpos[k0 + c] = qpos[p];
                qpos[p] = t0;
            }
            naff = 0;
        }
        __syncthreads();
        for (int i = tid; i < np; i += nt)
            if (qpos[i] != i) aff[atomicAdd(&naff, 1)] = i;
        __syncthreads();
        const int na = naff;
        {
            const int rv = tid < na ? rowperm[qpos[aff[tid]]] : 0;
            __syncthreads();
            if (tid < na) rowperm[aff[tid]] = rv;
        }
        // owned columns other than this panel: interchanges, rows K saved, rank-NB update
        for (int s = warp; s < ncol; s += GJI_W) {
            if (rank == owner && s / GJI_NB == ql) continue;
            float* col = Aown + (size_t)s * np;
            float v0 = 0.f, v1 = 0.f;
            if (lane < na) v0 = col[qpos[aff[lane]]];
            if (lane + 32 < na) v1 = col[qpos[aff[lane + 32]]];
            __syncwarp();
            if (lane < na) col[aff[lane]] = v0;
            if (lane + 32 < na) col[aff[lane + 32]] = v1;
            __syncwarp();
            if (lane < b) Tt[(size_t)lane * ncol + s] = col[k0 + lane];
        }
        __syncthreads();
        {
            // col[r] += sum_c Pt[c][r] T[c][s]: 4 x 4 register tiles (rows x slots)
            const int ntr = (np + 3) / 4, nts = (ncol + 3) / 4;
            for (int t = tid; t < ntr * nts; t += nt) {
                const int ts = t / ntr, r = (t - ts * ntr) * 4, s0 = ts * 4;
                bool skip[4];
                float acc[4][4];
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int s = s0 + y;
                    skip[y] = s >= ncol || (rank == owner && s / GJI_NB == ql);
#pragma unroll
                    for (int xx = 0; xx < 4; ++xx) acc[xx][y] = 0.f;
                }
                for (int c = 0; c < b; ++c) {
                    const float4 p4 = *reinterpret_cast<const float4*>(&Pt[(size_t)c * np + r]);
                    float tv[4];
#pragma unroll
                    for (int y = 0; y < 4; ++y) tv[y] = (s0 + y < ncol) ? Tt[(size_t)c * ncol + s0 + y] : 0.f;
                    const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                    for (int xx = 0; xx < 4; ++xx)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[xx][y] += pv[xx] * tv[y];
                }
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    if (skip[y]) continue;
                    float* col = Aown + (size_t)(s0 + y) * np;
#pragma unroll
                    for (int xx = 0; xx < 4; ++xx)
                        if (r + xx < np) col[r + xx] += acc[xx][y];
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    // column i of the storage is column rowperm[i] of the inverse
    for (int s = warp; s < ncol; s += GJI_W) {
        const int i = ((s / GJI_NB) * CL + rank) * GJI_NB + (s % GJI_NB);
        if (i >= np) continue;
        float* dst = Ainv + (size_t)rowperm[i] * np;
        for (int r = lane; r < np; r += 32) dst[r] = Aown[(size_t)s * np + r];
    }
    if (singular && tid == 0) atomicOr(status, ST_SINGULAR);
}

size_t lu_smem(int np, int xch) {
    const int npan = (np + GJ_NB - 1) / GJ_NB;
    const int ncmax = ((npan + LU_CL_MIN - 1) / LU_CL_MIN) * GJ_NB;   // the larger of the two cluster sizes' needs
    const size_t up = std::max((size_t)GJ_NB * ncmax, (size_t)np);
    const size_t xs = std::max((size_t)GJ_NB * ncmax, (size_t)xch * np);
    if (np > 2 * GJ_THREADS) return (size_t)-1;   // two panel rows per thread at most
    return sizeof(float) * ((size_t)GJ_NB * np + xs + up + PUB_FLOATS) +
           sizeof(int) * ((size_t)np + ncmax + np + 2 * GJ_NB_WARPS + np) + 16;
}


// Gauss-Jordan slab inverses (k_gj_inverse) for slabs of at most GJI_T
// unknowns: the largest cluster (8, 4, 2 CTAs) whose clusters for all the
// launch's slabs fit on the GPU at once (occupancy query on the first launch
// of a configuration, kept).
static cudaError_t gj_inverse(const IfPtrs& I, const ElimDev* el, int nel, int* status, cudaStream_t s) {
    static int fits[3] = {-1, -1, -1};
    static size_t fit_smem[3] = {0, 0, 0};
    static size_t set_smem = 0;
    const int cls[3] = {8, 4, 2};
    int cl = 2;
    for (int t = 0; t < 3; ++t) {
        const size_t smem = gji_smem(I.npad, cls[t]);
        if (smem > set_smem) {
            cudaError_t e = cudaFuncSetAttribute(k_gj_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            set_smem = smem;
        }
        if (fits[t] < 0 || fit_smem[t] != smem) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cls[t]);
            cfg.blockDim = dim3(GJI_T);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cls[t];
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_gj_inverse, &cfg) != cudaSuccess) {
                (void)cudaGetLastError();
                n = 0;
            }
            fits[t] = n;
            fit_smem[t] = smem;
        }
        if (nel <= fits[t]) {
            cl = cls[t];
            break;
        }
    }
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel, &status};
    return launch_cluster((const void*)k_gj_inverse, nel * cl, GJI_T, gji_smem(I.npad, cl), s, args, cl);
}

// Slab inverses of one elimination level.  variant 0: blocked Gauss-Jordan
// where the slabs are small enough (else the LU); 1: the LU with inverse
// columns; 2: register-resident Gauss-Jordan (slab_gjr.cu) where the slabs
// are small enough (else the LU).
int slab_inverse_gj_ok(int npad) { return npad <= GJI_T; }
int slab_inverse_gjr_npad(int npad);
cudaError_t gjr_inverse(const IfPtrs& I, const ElimDev* el, int nel, int* status, cudaStream_t s);

cudaError_t lu_inverse(const IfPtrs& I, const ElimDev* el, int nel, int* status, int variant, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    if (variant == 2 && slab_inverse_gjr_npad(I.npad)) return gjr_inverse(I, el, nel, status, s);
    if (variant == 0 && I.npad <= GJI_T) return gj_inverse(I, el, nel, status, s);
    const size_t smem = lu_smem(I.npad, I.xch);
    // panel rows per thread: one for slabs of up to GJ_THREADS unknowns, else two
    const bool two = I.npad > GJ_THREADS;
    const void* kern = two ? (const void*)k_lu_inverse<2> : (const void*)k_lu_inverse<1>;
    static size_t set_smem[2] = {0, 0};
    if (smem > set_smem[two]) {
        cudaError_t e = two ? cudaFuncSetAttribute(k_lu_inverse<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(k_lu_inverse<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_smem[two] = smem;
    }
    // 8-CTA clusters when the launch's slabs all fit at once (the query runs
    // on the first, eager launch of a configuration and is kept)
    static int max8[2] = {-1, -1};
    static size_t max8_smem[2] = {0, 0};
    if (max8[two] < 0 || max8_smem[two] != smem) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(LU_CL_MAX);
        cfg.blockDim = dim3(GJ_THREADS);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = LU_CL_MAX;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            n = 0;
        }
        max8[two] = n;
        max8_smem[two] = smem;
    }
    const int cl = nel <= max8[two] ? LU_CL_MAX : LU_CL_MIN;
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel, &status};
    return launch_cluster(kern, nel * cl, GJ_THREADS, smem, s, args, cl);
}

size_t elim_smem_bytes(int nmv, int cw) {
    // Asm (nmv4^2) + stL, stQ (32 (nmv4 + 4) each) + Csm (nmv4 cw4), with nmv4 / cw4 rounded up to 4
    const size_t n4 = ((size_t)nmv + 3) & ~size_t(3), c4 = ((size_t)cw + 3) & ~size_t(3);
    return sizeof(float) * (n4 * n4 + 64 * (n4 + 4) + n4 * c4) + 16;
}

cudaError_t bcr_elim(const IfPtrs& I, const ElimDev* el, int nel, size_t smem, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    static size_t set_smem = 0;
    if (smem > set_smem) {
        cudaError_t e = cudaFuncSetAttribute(k_bcr_elim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bcr_elim, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        set_smem = smem;
    }
    // the upper levels eliminate few slabs: more CTAs per slab (row chunks of
    // the four products) while the level's clusters fit on the GPU at once
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int cl = nel * 16 <= nsm ? 16 : nel * 8 <= nsm ? 8 : GJ_CL;
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel};
    return launch_cluster((const void*)k_bcr_elim, nel * cl, EL_THREADS, smem, s, args, cl);
}
