// 2D local Robin/Darcy solves of MRCM-OS on sm_103a.
//
// One CTA per job (a subdomain box).  The cell-centred RT0 operator of the
// box (Sec. 2.2; interior faces T = a 2 K_L K_R / (h (K_L + K_R)), Robin faces
// T = a / (h / 2K + beta) with beta = alpha H / K_H, Dirichlet T = 2 a K / h)
// is block tridiagonal over grid lines of b <= 32 cells.  It is factored once
// (Algorithm 1, Steps 1 and 6) as a block LDL^T whose pivots are the line
// Schur complements S_j = T_j - C_{j-1} S_{j-1}^{-1} C_{j-1}; each S_j is
// inverted in registers by one warp (Gauss-Jordan, SPD so no pivoting) and
// the inverses are kept.  A solve is then two sweeps of dense b x b
// mat-vecs, one warp per right-hand side (Steps 2, 4, 7).
//
// Precision: T = double is the FP64 form.  T = float is the mixed form: the
// operator is Jacobi scaled, the Schur diagonals and every Gauss-Jordan
// pivot reciprocal are formed in FP64, the sweeps run in FP32, and each
// right-hand side is refined with FP64 residuals of the unscaled operator
// until |r|_inf <= ir_tol |b|_inf.
//
// FP64 division and square root are avoided in the hot loops (GB300 has a
// narrow FP64 pipe): face transmissibilities come precomputed per problem,
// reciprocals are an FP32 seed refined by two FP64 Newton steps, and the
// Jacobi scale is an FP32 rsqrt used consistently on both sides.

#include "box2d.cuh"


// ---------------------------------------------------------------------------
// Steps 1, 2, 4 and 6 of Algorithm 1 for 2D subdomains.
// ---------------------------------------------------------------------------
template <typename T, int BW, bool EX>
__global__ void __launch_bounds__(NWARP * 32, 1) k_local2d(DevPtrs P, MethodDev Mth, const Job* jobs) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool mixed = std::is_same<T, float>::value;
    const Job job = jobs[blockIdx.x];
    const SubDev sd = P.sub[job.item];
    const MemberDev& md = P.mem[sd.member];
    __shared__ Box B;
    if (threadIdx.x == 0) {
        if (job.type == JOB_PART) setup_box(B, md, sd.lo, sd.hi, Mth.alpha_b);
        else setup_box(B, md, sd.loh, sd.hih, job.type == JOB_SFACT ? Mth.alpha_s : Mth.alpha_b);
    }
    __syncthreads();
    // right-hand sides: the basis functions, or the particular problem on
    // Omega_i; with the particular problem on hat-Omega_i (a variant) it is
    // the basis job's last right-hand side, k = nbasis, its vector kept in
    // global memory (the basis box has no shared memory left for it)
    const bool hat_part = job.type == JOB_BASIS && Mth.part_hat;
    const int nrhs = job.type == JOB_BASIS ? sd.nbasis + (hat_part ? 1 : 0) : (job.type == JOB_PART ? 1 : 0);
    Carve<T> C = carve<T>(smem, B.nx, B.ny, nrhs > 0 ? min(nrhs, NWARP) : 1, job.type == JOB_PART);
    if (!mrcm_check(P.status, C.end <= mrcm_dyn_smem_bytes(), 1, (long long)C.end)) return;   // uniform
    if (threadIdx.x == 0) { C.flags[0] = 0; C.flags[1] = 0; }
    build_ops(B, md, P, C.O);
    fill_scale(B, C.O, mixed);
    if (mixed) scale_ops(B, C.O);   // D A D: the factor and the refinement work in scaled variables
    factor_box<T, BW, EX, mixed>(B, C.O, C.Sinv, C.cys, C.cxs, &C.flags[0]);

    // keep the factor for the smoothing steps, as the subdomain's smoothing pack
    const bool keep = (job.type == JOB_SFACT) || (job.type == JOB_BASIS && Mth.same_alpha);
    if (keep) {
        unsigned char* pk = (unsigned char*)((T*)P.fac + (size_t)job.item * P.fac_stride);
        const SPack L = spack_layout(B.nx, B.ny, sizeof(T));
        T* dst = (T*)pk;
        const size_t nS = sinv_len(B.nx, B.ny, sizeof(T));
        for (size_t t = threadIdx.x; t < nS; t += blockDim.x) dst[t] = C.Sinv[t];
        double* dd = P.dsc + (size_t)job.item * P.dsc_stride;
        const double* fk = P.f + md.cell_off;
        const double vk = md.h[0] * md.h[1];
        for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
            dd[c] = C.O.dsc[c];
            ((double*)(pk + L.cd))[c] = C.O.cd[c];
            ((double*)(pk + L.cx))[c] = C.O.cx[c];
            ((double*)(pk + L.cy))[c] = C.O.cy[c];
            ((double*)(pk + L.dsc))[c] = C.O.dsc[c];
            ((double*)(pk + L.bst))[c] =
                C.O.dsc[c] * source_rhs(B, C.O, fk, md.n[0], vk, md.h[1], md.h[0], nullptr, c % B.nx, c / B.nx);
            ((T*)(pk + L.cys))[c] = C.cys[c];
        }
        for (int t = threadIdx.x; t < 2 * (B.nx + B.ny); t += blockDim.x) {
            ((double*)(pk + L.bT))[t] = C.O.bT[t];
            ((double*)(pk + L.bB))[t] = C.O.bB[t];
        }
    }
    if (C.flags[0] && threadIdx.x == 0) {
        atomicOr(&P.status[0], ST_NOT_SPD);
        atomicExch(&P.status[2], job.item);
    }
    if (nrhs == 0) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* zb = C.zbuf + warp * 64;
    const int npsi = Mth.npsi;
    const double vol = md.h[0] * md.h[1];
    const double ax = md.h[1], ay = md.h[0];
    const double rax = 1.0 / ax, ray = 1.0 / ay;
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int offx = sd.lo[0] - B.lo[0], offy = sd.lo[1] - B.lo[1];
    int maxit = 0, nsolve = 0;
    const double* fm = P.f + md.cell_off;
    for (int k = warp; k < nrhs; k += NWARP) {
        double* x = C.X + (size_t)warp * B.n;
        T* w = C.W + (size_t)warp * B.n;
        int it;
        int sk = -1, mk = 0;
        const bool part = job.type == JOB_PART || k >= sd.nbasis;   // the particular problem
        if (!part) {
            // k -> (side, m): sides of Gamma_i in increasing id, npsi functions each
            int q = k / npsi;
            mk = k % npsi;
            for (int sid = 0; sid < 4; ++sid)
                if (sd.side_mask & (1 << sid)) {
                    if (q == 0) { sk = sid; break; }
                    --q;
                }
            if constexpr (mixed) {
                // b~ on the Robin side: lane pos holds that of face pos
                const int len = (sk >> 1) == 0 ? B.ny : B.nx;
                double mine = 0.0;
                if (lane < len) {
                    const int ci = (sk >> 1) == 0 ? lane * B.nx + (sk == 0 ? 0 : B.nx - 1)
                                                  : (sk == 2 ? 0 : (B.ny - 1) * B.nx) + lane;
                    mine = C.O.dsc[ci] * C.O.bT[side_off(B, sk) + lane] * psi_val(mk, lane, len, B.rlen[sk]);
                }
                RhsScSide rb{sk, mine};
                it = warp_solve_sc<RhsScSide, EX ? BW : 0>(B, C.O, C.Sinv, C.cys, x, w, zb, rb, Mth.ir_tol,
                                                            Mth.max_ir, &C.flags[1]);
            } else {
                RhsBasis rb{sk, mk};
                it = warp_solve<T, RhsBasis>(B, C.O, C.Sinv, C.cys, x, w, zb, rb, Mth.ir_tol, Mth.max_ir,
                                             &C.flags[1]);
            }
        } else {
            // the particular problem: fixed right-hand side staged once (b~ in the mixed form)
            double* bs = hat_part ? P.bsrc + (size_t)job.item * P.dsc_stride : C.bsrc;
            for (int c = lane; c < B.n; c += 32) {
                const int i = c % B.nx, j = c / B.nx;
                bs[c] = C.O.dsc[c] * source_rhs(B, C.O, fm, md.n[0], vol, ax, ay, nullptr, i, j);
            }
            __syncwarp();
            if constexpr (mixed) {
                RhsScStored rs{bs};
                it = warp_solve_sc<RhsScStored, EX ? BW : 0>(B, C.O, C.Sinv, C.cys, x, w, zb, rs, Mth.ir_tol,
                                                              Mth.max_ir, &C.flags[1]);
            } else {
                RhsStored rs{bs};
                it = warp_solve<T, RhsStored>(B, C.O, C.Sinv, C.cys, x, w, zb, rs, Mth.ir_tol, Mth.max_ir,
                                              &C.flags[1]);
            }
        }
        if constexpr (mixed) {
            // back from the scaled iterate
            for (int c = lane; c < B.n; c += 32) x[c] *= C.O.dsc[c];
        }
        maxit = max(maxit, it);
        nsolve += it;
        __syncwarp();
        // ---- outputs: restriction to Omega_i and Gamma_i traces (Eq. (informed_space)) ----
        const int slot = !part ? k : P.nbasis_max;
        double* psi_out = !part
                              ? P.Psi + ((size_t)job.item * P.nbasis_max + k) * P.ncell_i_max
                              : P.pbar + (size_t)job.item * P.ncell_i_max;
        for (int c = lane; c < nIx * nIy; c += 32) {
            const int i = c % nIx, j = c / nIx;
            psi_out[c] = x[(j + offy) * B.nx + (i + offx)];
        }
        double* mom = P.mom + (((size_t)job.item * (P.nbasis_max + 1) + slot) * MRCM_MAXSIDE) * npsi * 2;
        for (int sid = 0; sid < 4; ++sid) {
            if (!(sd.side_mask & (1 << sid))) continue;
            const int a = sid >> 1;
            const int len = a == 0 ? nIy : nIx;
            const double rl = 1.0 / (double)len;
            const double area = a == 0 ? ax : ay;
            const double rarea = a == 0 ? rax : ray;
            double* ug = !part
                             ? P.Ug + (((size_t)job.item * P.nbasis_max + k) * MRCM_MAXSIDE + sid) * P.side_max
                             : P.ubg + ((size_t)job.item * MRCM_MAXSIDE + sid) * P.side_max;
            double fmv[3] = {0, 0, 0}, pmv[3] = {0, 0, 0};
            for (int e = lane; e < len; e += 32) {
                int i, j;
                if (a == 0) { j = offy + e; i = (sid == 0) ? offx : offx + nIx - 1; }
                else        { i = offx + e; j = (sid == 2) ? offy : offy + nIy - 1; }
                const int cL = j * B.nx + i;
                const double pL = x[cL];
                const long long gL = md.cell_off + (B.lo[0] + i) + (long long)md.n[0] * (B.lo[1] + j);
                const double hkL = P.hk[gL * 3 + a];
                // interior face transmissibility (unscaled) from the face coefficients
                bool inner;
                int cR;
                double Tf;
                if (sid == 0) { inner = i > 0; cR = cL - 1; Tf = inner ? P.Tf[(gL - 1) * 3 + 0] : 0; }
                else if (sid == 1) { inner = i < B.nx - 1; cR = cL + 1; Tf = inner ? P.Tf[gL * 3 + 0] : 0; }
                else if (sid == 2) { inner = j > 0; cR = cL - B.nx; Tf = inner ? P.Tf[(gL - md.n[0]) * 3 + 1] : 0; }
                else { inner = j < B.ny - 1; cR = cL + B.nx; Tf = inner ? P.Tf[gL * 3 + 1] : 0; }
                double uo, pi;
                if (inner) {
                    uo = Tf * (pL - x[cR]) * rarea;
                    pi = pL - uo * hkL;
                } else {
                    // Robin face of the box (l = 0 basis, or the particular problem)
                    const int pos = a == 0 ? j : i;
                    const int blen = a == 0 ? B.ny : B.nx;
                    double lam = 0.0;
                    if (!part && sid == sk) lam = psi_val(mk, pos, blen, B.rlen[sid]);
                    uo = C.O.bT[side_off(B, sid) + pos] * (pL - lam) * rarea;
                    if (job.type == JOB_PART) pi = C.O.bB[side_off(B, sid) + pos] * uo;  // beta ubar.n
                    else pi = pL - uo * hkL;
                }
                ug[e] = uo;
                for (int m = 0; m < npsi; ++m) {
                    const double ps = psi_val(m, e, len, rl);
                    fmv[m] += ps * uo * area;
                    pmv[m] += area * ps * pi;
                }
            }
            for (int m = 0; m < npsi; ++m) {
                for (int o = 16; o; o >>= 1) {
                    fmv[m] += __shfl_xor_sync(0xffffffffu, fmv[m], o);
                    pmv[m] += __shfl_xor_sync(0xffffffffu, pmv[m], o);
                }
                if (lane == 0) {
                    mom[(sid * npsi + m) * 2 + 0] = fmv[m];
                    mom[(sid * npsi + m) * 2 + 1] = pmv[m];
                }
            }
        }
    }
    if (lane == 0 && maxit > 0) {
        atomicMax(&P.status[1], maxit);
        atomicAdd(&P.status[3], nsolve);
    }
    __syncthreads();
    if (threadIdx.x == 0 && C.flags[1]) atomicOr(&P.status[0], ST_NO_CONV);
}

// ---------------------------------------------------------------------------
// Step 7: one colour phase of a smoothing step (Sec. 3, Eqs. (sm_1)-(sm_2)).
// One CTA (SM_WARPS warps) per subdomain of the colour; the kept factor is
// staged into shared memory by the bulk-copy (TMA) engine while the
// coefficients and Robin data are formed; the whole CTA runs the sweeps
// (each line's product split over the warps) and the FP64 residuals.
// ---------------------------------------------------------------------------
constexpr int SM_WARPS = 4;

template <typename T>
__global__ void __launch_bounds__(SM_WARPS * 32) k_smooth2d(DevPtrs P, MethodDev Mth, const int* items) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool mixed = std::is_same<T, float>::value;
    const int item = items[blockIdx.x];
    const SubDev sd = P.sub[item];
    const MemberDev& md = P.mem[sd.member];
    __shared__ Box B;
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t never;   // failure-detection test only: a barrier nothing arrives at
    if (threadIdx.x == 0) setup_box(B, md, sd.loh, sd.hih, Mth.alpha_s);
    __syncthreads();
    const size_t n = (size_t)B.n;
    // the smoothing pack (factor, operator, fixed right-hand side) first, by one bulk copy
    const SPack L = spack_layout(B.nx, B.ny, sizeof(T));
    T* Sinv = (T*)smem;
    Ops O;
    O.cd = (double*)(smem + L.cd);
    O.cx = (double*)(smem + L.cx);
    O.cy = (double*)(smem + L.cy);
    O.dsc = (double*)(smem + L.dsc);
    O.hk = nullptr;
    O.bT = (double*)(smem + L.bT);
    O.bB = (double*)(smem + L.bB);
    double* bsrc = (double*)(smem + L.bst);   // fixed part, then the Robin terms of this step
    T* cys = (T*)(smem + L.cys);
    size_t o = L.bytes;
    auto take = [&](size_t bytes) { unsigned char* p = smem + o; o += align16(bytes); return p; };
    double* lam = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    double* lun = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    T* zbuf = (T*)take(sizeof(T) * 32 * SM_WARPS);       // line input of the sweeps
    T* red = (T*)take(sizeof(T) * 2 * 32 * SM_WARPS);    // partial sums of the warps (FP64 sweeps), two line parities
    unsigned int* nrm = (unsigned int*)take(16);
    double* x = (double*)take(sizeof(double) * n);
    T* w = mixed ? (T*)take(sizeof(T) * n) : (T*)x;
    int* flags = (int*)take(64);
    if (!mrcm_check(P.status, o <= mrcm_dyn_smem_bytes(), 2, (long long)o)) return;   // uniform
    const uint32_t pbytes = (uint32_t)L.bytes;
    const unsigned char* Pg = (const unsigned char*)((const T*)P.fac + (size_t)item * P.fac_stride);
    if (threadIdx.x == 0) {
        flags[0] = 0;
        flags[1] = 0;
        mbar_init(&bar, 1);
        if (Mth.wait0 > 0) mbar_init(&never, 1);
        mbar_expect_tx(&bar, pbytes);
        // a bulk copy needs 16-byte aligned ends and a size that is a multiple of 16
        if (mrcm_check(P.status, ((uintptr_t)Pg & 15) == 0 && (pbytes & 15) == 0 && pbytes <= L.bytes, 3,
                       (long long)pbytes))
            bulk_g2s(smem, Pg, pbytes, &bar);
    }
    // launched as a programmatic dependent of the previous colour: the pack
    // (written by the basis kernel, two or more launches earlier) is in flight
    // already; the state is read only once the previous launch is complete
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // Robin data from the current solution, while the pack is in flight:
    // lambda = -beta u.n + pi with n the outward normal of hat-Omega_i and
    // pi = p - u.n h / (2K) of the cell inside
    const double* pst = P.p + md.cell_off;
    const double* ust = P.u + md.cell_off * 4;
    const double* hkg = P.hk + md.cell_off * 3;
    for (int sid = 0; sid < 4; ++sid) {
        if (B.kind[sid] != 2) continue;
        const int a = sid >> 1;
        const int len = a == 0 ? B.ny : B.nx;
        for (int pos = threadIdx.x; pos < len; pos += blockDim.x) {
            int i, j;
            if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; }
            else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; }
            const long long g = (B.lo[0] + i) + (long long)md.n[0] * (B.lo[1] + j);
            const double un = ust[g * 4 + sid];
            lun[side_off(B, sid) + pos] = un;
            lam[side_off(B, sid) + pos] = pst[g] - un * hkg[g * 3 + a];
        }
    }
    // mixed form: the refinement starts from the current pressure on the box
    // (read now; scaled once the pack, with D, has arrived)
    if (mixed)
        for (int c = threadIdx.x; c < B.n; c += blockDim.x)
            x[c] = pst[(B.lo[0] + c % B.nx) + (long long)md.n[0] * (B.lo[1] + c / B.nx)];
    // the unscaled face transmissibilities the output needs (shared memory holds D A D), read while the pack
    // is in flight: this thread's cells of Omega_i, faces x-, x+, y-, y+ (two cells per thread at most)
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int offx = sd.lo[0] - B.lo[0], offy = sd.lo[1] - B.lo[1];
    const double* Tfg = P.Tf + md.cell_off * 3;
    double tfo[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int c = threadIdx.x + q * blockDim.x;
        const int i = c % nIx + offx, j = c / nIx + offy;
        const long long g = (B.lo[0] + i) + (long long)md.n[0] * (B.lo[1] + j);
        const bool ok = c < nIx * nIy;
        tfo[q][0] = (ok && i > 0) ? Tfg[(g - 1) * 3 + 0] : 0.0;
        tfo[q][1] = (ok && i < B.nx - 1) ? Tfg[g * 3 + 0] : 0.0;
        tfo[q][2] = (ok && j > 0) ? Tfg[(g - md.n[0]) * 3 + 1] : 0.0;
        tfo[q][3] = (ok && j < B.ny - 1) ? Tfg[g * 3 + 1] : 0.0;
    }
    int it = 0;
    // every thread reads the staged pack: all wait for the copy, and agree on a late one
    // (with the failure-detection test's wait set, the first wait is for a
    // barrier nothing arrives at, for that many cycles: it runs out)
    const bool arrived = Mth.wait0 > 0 ? mbar_wait(&never, 0, Mth.wait0) : mbar_wait(&bar, 0);
    if (!__syncthreads_or(!arrived)) {
        for (int sid = 0; sid < 4; ++sid) {
            if (B.kind[sid] != 2) continue;
            const int len = (sid >> 1) == 0 ? B.ny : B.nx;
            for (int pos = threadIdx.x; pos < len; pos += blockDim.x)
                lam[side_off(B, sid) + pos] -= O.bB[side_off(B, sid) + pos] * lun[side_off(B, sid) + pos];
        }
        __syncthreads();
        // Robin terms of the right-hand side, one side at a time (corner cells lie on two)
        for (int sid = 0; sid < 4; ++sid) {
            if (B.kind[sid] != 2) continue;
            const int a = sid >> 1;
            const int len = a == 0 ? B.ny : B.nx;
            for (int pos = threadIdx.x; pos < len; pos += blockDim.x) {
                const int i = a == 0 ? ((sid == 0) ? 0 : B.nx - 1) : pos;
                const int j = a == 0 ? pos : ((sid == 2) ? 0 : B.ny - 1);
                const int c = j * B.nx + i;
                bsrc[c] += O.dsc[c] * (O.bT[side_off(B, sid) + pos] * lam[side_off(B, sid) + pos]);
            }
            __syncthreads();
        }
        if constexpr (mixed) {
            // the scaled start x~ = D^-1 x (an FP32 reciprocal of the FP32 scale: a start only)
            for (int c = threadIdx.x; c < B.n; c += blockDim.x)
                x[c] *= f2d_bits(__frcp_rn(d2f_bits(O.dsc[c])));
            __syncthreads();
            it = cta_solve_sc(B, O, (const float*)Sinv, (const float*)cys, x, (float*)w, (float*)zbuf, nrm, bsrc,
                              Mth.ir_tol, Mth.max_ir, &flags[0], true);
            for (int c = threadIdx.x; c < B.n; c += blockDim.x) x[c] *= O.dsc[c];
            __syncthreads();
        } else {
            RhsStored rs{bsrc};
            it = cta_solve<T>(B, O, Sinv, cys, x, w, zbuf, red, nrm, rs, Mth.ir_tol, Mth.max_ir, &flags[0], false);
        }
    } else if (threadIdx.x == 0) {
        flags[1] = 1;
    }
    __syncthreads();
    if (flags[1]) {
        // the staged factor never arrived: report, wait once more for the copy
        // in flight (bounded) so that no copy targets a finished CTA, and stop
        if (threadIdx.x == 0) {
            atomicOr(&P.status[0], ST_BAD);
            mbar_wait(&bar, 0);
        }
        __syncthreads();
        return;
    }
    // overwrite (u, p) on Omega_i with the restriction
    double* pw = P.p + md.cell_off;
    double* uw = P.u + md.cell_off * 4;
    const double rax = 1.0 / md.h[1], ray = 1.0 / md.h[0];
    for (int q = 0, c = threadIdx.x; c < nIx * nIy; ++q, c += blockDim.x) {
        const int i = c % nIx + offx, j = c / nIx + offy;
        const int cl = j * B.nx + i;
        const long long g = (B.lo[0] + i) + (long long)md.n[0] * (B.lo[1] + j);
        if (!mrcm_check(P.status, g >= 0 && g < (long long)md.n[0] * md.n[1], 4, g)) continue;
        const double pc = x[cl];
        pw[g] = pc;
        // transmissibilities: prefetched for a thread's first two cells, else read here
        double tf[4];
        if (q < 2) {
#pragma unroll
            for (int sid = 0; sid < 4; ++sid) tf[sid] = q == 0 ? tfo[0][sid] : tfo[1][sid];
        } else {
            tf[0] = i > 0 ? Tfg[(g - 1) * 3 + 0] : 0.0;
            tf[1] = i < B.nx - 1 ? Tfg[g * 3 + 0] : 0.0;
            tf[2] = j > 0 ? Tfg[(g - md.n[0]) * 3 + 1] : 0.0;
            tf[3] = j < B.ny - 1 ? Tfg[g * 3 + 1] : 0.0;
        }
        double uo[4];
        for (int sid = 0; sid < 4; ++sid) {
            const int a = sid >> 1;
            const double rarea = a == 0 ? rax : ray;
            const bool edge = (sid == 0 && i == 0) || (sid == 1 && i == B.nx - 1) || (sid == 2 && j == 0) ||
                              (sid == 3 && j == B.ny - 1);
            if (!edge) {
                const int cn = sid == 0 ? cl - 1 : sid == 1 ? cl + 1 : sid == 2 ? cl - B.nx : cl + B.nx;
                uo[sid] = tf[sid] * (pc - x[cn]) * rarea;
            } else {
                const int pos = a == 0 ? j : i;
                const double Tb = O.bT[side_off(B, sid) + pos];
                if (B.kind[sid] == 2) uo[sid] = Tb * (pc - lam[side_off(B, sid) + pos]) * rarea;
                else if (B.kind[sid] == 1) uo[sid] = Tb * (pc - B.val[sid]) * rarea;
                else uo[sid] = B.val[sid];
            }
        }
        for (int sid = 0; sid < 4; ++sid) uw[g * 4 + sid] = uo[sid];
    }
    if (threadIdx.x == 0) {
        atomicMax(&P.status[1], it);
        atomicAdd(&P.status[3], it);
        if (flags[0]) atomicOr(&P.status[0], ST_NO_CONV);
    }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
size_t local2d_smem(int prec, int nx, int ny, int nrhs, bool part) {
    return prec == 0 ? carve_bytes<double>(nx, ny, nrhs, part) : carve_bytes<float>(nx, ny, nrhs, part);
}

size_t spack_bytes(int prec, int nx, int ny) {
    return spack_layout(nx, ny, prec == 0 ? sizeof(double) : sizeof(float)).bytes;
}

size_t smooth2d_smem(int prec, int nx, int ny) {
    const size_t n = (size_t)nx * ny;
    const size_t tsz = prec == 0 ? sizeof(double) : sizeof(float);
    size_t s = spack_bytes(prec, nx, ny);
    s += align16(sizeof(double) * 2 * (nx + ny)) * 2;
    s += align16(tsz * 32 * SM_WARPS) + align16(tsz * 2 * 32 * SM_WARPS) + 16;
    s += align16(sizeof(double) * n);
    if (prec != 0) s += align16(tsz * n);
    return s + 64;
}

template <typename T, int BW, bool EX>
static cudaError_t launch_local_t(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs,
                                  size_t smem, cudaStream_t s) {
    auto kern = k_local2d<T, BW, EX>;
    static size_t set_smem = 0;
    if (smem > set_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // all of the unified L1 / shared storage as shared memory (two CTAs per SM)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        set_smem = smem;
    }
    kern<<<njobs, NWARP * 32, smem, s>>>(P, M, jobs);
    return cudaGetLastError();
}

// Job classes: local2d_class(prec, nx).  The FP32 form has one kernel per line
// width that is a multiple of 4 (width known at compile time: its line
// inversions and sweeps run without width guards); other widths, and the
// FP64 form, run a kernel for widths up to 8, 16, 24 or 32.
int local2d_class(int prec, int nx) {
    if (prec != 0 && nx % 4 == 0 && nx <= 32) return nx;
    return 100 + (nx <= 8 ? 8 : nx <= 16 ? 16 : nx <= 24 ? 24 : 32);
}

cudaError_t launch_local2d(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs, int cls,
                           size_t smem, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    if (M.prec == 0) {
        if (cls <= 108) return launch_local_t<double, 8, false>(P, M, jobs, njobs, smem, s);
        if (cls <= 116) return launch_local_t<double, 16, false>(P, M, jobs, njobs, smem, s);
        if (cls <= 124) return launch_local_t<double, 24, false>(P, M, jobs, njobs, smem, s);
        return launch_local_t<double, 32, false>(P, M, jobs, njobs, smem, s);
    }
    switch (cls) {
        case 4: return launch_local_t<float, 4, true>(P, M, jobs, njobs, smem, s);
        case 8: return launch_local_t<float, 8, true>(P, M, jobs, njobs, smem, s);
        case 12: return launch_local_t<float, 12, true>(P, M, jobs, njobs, smem, s);
        case 16: return launch_local_t<float, 16, true>(P, M, jobs, njobs, smem, s);
        case 20: return launch_local_t<float, 20, true>(P, M, jobs, njobs, smem, s);
        case 24: return launch_local_t<float, 24, true>(P, M, jobs, njobs, smem, s);
        case 28: return launch_local_t<float, 28, true>(P, M, jobs, njobs, smem, s);
        case 32: return launch_local_t<float, 32, true>(P, M, jobs, njobs, smem, s);
        default: break;
    }
    if (cls <= 108) return launch_local_t<float, 8, false>(P, M, jobs, njobs, smem, s);
    if (cls <= 116) return launch_local_t<float, 16, false>(P, M, jobs, njobs, smem, s);
    if (cls <= 124) return launch_local_t<float, 24, false>(P, M, jobs, njobs, smem, s);
    return launch_local_t<float, 32, false>(P, M, jobs, njobs, smem, s);
}

template <typename T>
static cudaError_t launch_smooth2d_t(const DevPtrs& P, const MethodDev& M, const int* items, int nitems, size_t smem,
                                     cudaStream_t s) {
    auto kern = k_smooth2d<T>;
    static size_t set_smem = 0;
    if (smem > set_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_smem = smem;
    }
    // programmatic dependent launch (see k_smooth2d): scheduled while the
    // previous kernel drains
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nitems);
    cfg.blockDim = dim3(SM_WARPS * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DevPtrs Pc = P;
    MethodDev Mc = M;
    void* args[] = {&Pc, &Mc, (void*)&items};
    return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
}

cudaError_t launch_smooth2d(const DevPtrs& P, const MethodDev& M, const int* items, int nitems, size_t smem,
                            cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    return M.prec == 0 ? launch_smooth2d_t<double>(P, M, items, nitems, smem, s)
                       : launch_smooth2d_t<float>(P, M, items, nitems, smem, s);
}
