// Reverse mode of the 2D MRCM-OS pipeline with respect to log K, on sm_103a.
//
// The method depends on K only through three face-coefficient arrays, the
// interior transmissibility Tf = a 2 K_L K_R / (h (K_L + K_R)), the cell
// terms h / (2K) and the face terms H / K_H (so that beta = alpha H / K_H and a
// Robin face has T = a / (h / 2K + beta)); Sec. 2.2 and Eq. (genRobin).  Every
// reverse kernel accumulates dL/d(those coefficients); k_grad_logK maps them
// to dL/dlog K at the end.
//
// For one box solve A p = b(lambda), u = V(p, lambda) with seeds (gp, gu) the
// adjoint is mu = A^{-1} (gp + dV/dp^T gu) -- the same factor, A is SPD -- and
// dL/dc = -mu^T (dA/dc) p + mu^T db/dc + gu . dV/dc per face coefficient c.
// The forward solution p is recomputed from the kept factor instead of
// being stored.
//
// Kernels, in the order the host issues them:
//   k_adj_smooth2d    one colour pass of a smoothing step backwards
//                     (Eqs. (sm_1)-(sm_2)), colours and steps in reverse order
//   k_adj_assemble2d  the superposition of Eqs. (addu), (addp) backwards
//   (interface.cu)    dL/drhs = G^-T dL/dX, the interface system transposed
//   k_adj_moments     dL/d(flux and pressure moments) from dL/dG, dL/drhs
//   k_adj_local2d     basis problems (Eq. (oversampling_problem)) and
//                     particular problems (Eqs. (111dbar)-(122dbar)) backwards
//   k_grad_logK       face-coefficient adjoints -> dL/dlog K
#include "box2d.cuh"

namespace {

constexpr int AS_WARPS = 4;   // k_adj_smooth2d: warp 0 solves, all warps form data

// row of test function m on side `sid` of its owner (flux rows of the high
// sides first, then pressure rows of the low sides; same order as
// k_if_assemble)
__device__ int row_pos(const SubDev& o, int d, int npsi, int kind, int sid, int m) {
    int q = 0;
    for (int a = 0; a < d; ++a) {
        const int sh = 2 * a + 1;
        if (o.side_mask & (1 << sh)) {
            if (kind == 0 && sh == sid) return q + m;
            q += npsi;
        }
    }
    for (int a = 0; a < d; ++a) {
        const int sl = 2 * a;
        if (o.side_mask & (1 << sl)) {
            if (kind == 1 && sl == sid) return q + m;
            q += npsi;
        }
    }
    return -1;
}

}  // namespace

// ---------------------------------------------------------------------------
// One colour pass of a smoothing step, backwards.  One CTA per subdomain of
// the colour.  Forward: lambda from the recorded state on d hat-Omega_i \ d
// Omega, a solve on hat-Omega_i with the sources, overwrite of (p, u) on
// Omega_i.  Backward: the seeds on Omega_i are taken (and cleared), the
// forward solution is recomputed, one adjoint solve, and dL/dlambda is
// passed on to the recorded state.  Subdomains of one colour have disjoint
// oversampled boxes (2 l < H), so their writes never meet.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(AS_WARPS * 32) k_adj_smooth2d(DevPtrs P, MethodDev Mth, AdjPtrs A,
                                                                const int* items) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool mixed = std::is_same<T, float>::value;
    const int item = items[blockIdx.x];
    const SubDev sd = P.sub[item];
    const MemberDev& md = P.mem[sd.member];
    __shared__ Box B;
    if (threadIdx.x == 0) setup_box(B, md, sd.loh, sd.hih, Mth.alpha_s);
    __syncthreads();
    const size_t n = (size_t)B.n;
    const int per = 2 * (B.nx + B.ny);
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = smem + o; o += align16(bytes); return p; };
    T* Sinv = (T*)take(sizeof(T) * sinv_len(B.nx, B.ny, sizeof(T)));
    Ops O;
    O.cd = (double*)take(sizeof(double) * n);
    O.cx = (double*)take(sizeof(double) * n);
    O.cy = (double*)take(sizeof(double) * n);
    O.dsc = (double*)take(sizeof(double) * n);
    O.hk = (double*)take(sizeof(double) * 2 * n);
    O.bT = (double*)take(sizeof(double) * per);
    O.bB = (double*)take(sizeof(double) * per);
    double* lam = (double*)take(sizeof(double) * per);
    double* rt = (double*)take(sizeof(double) * n);
    T* cys = (T*)take(sizeof(T) * n);
    T* zbuf = (T*)take(sizeof(T) * 64);   // two line inputs of the twisted sweeps
    double* x = (double*)take(sizeof(double) * n);
    double* mu = (double*)take(sizeof(double) * n);
    T* w = mixed ? (T*)take(sizeof(T) * n) : nullptr;
    double* su = (double*)take(sizeof(double) * 4 * n);
    int* flags = (int*)take(64);

    const T* Sg = (const T*)P.fac + (size_t)item * P.fac_stride;
    for (size_t t = threadIdx.x; t < sinv_len(B.nx, B.ny, sizeof(T)); t += blockDim.x) Sinv[t] = Sg[t];
    if (threadIdx.x == 0) flags[0] = 0;
    build_ops(B, md, P, O);
    const double* dd = P.dsc + (size_t)item * P.dsc_stride;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) O.dsc[c] = dd[c];
    __syncthreads();
    for (int c = threadIdx.x; c < B.n; c += blockDim.x)
        cys[c] = (T)(O.cy[c] * O.dsc[c] * ((c + B.nx < B.n) ? O.dsc[c + B.nx] : 0.0));
    const int nxg = md.n[0];
    const double* pst = A.ps + md.cell_off;
    const double* ust = A.us + md.cell_off * 4;
    for (int sid = 0; sid < 4; ++sid) {
        if (B.kind[sid] != 2) continue;
        const int a = sid >> 1;
        const int len = a == 0 ? B.ny : B.nx;
        for (int pos = threadIdx.x; pos < len; pos += blockDim.x) {
            int i, j;
            if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; }
            else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; }
            const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
            const double un = ust[g * 4 + sid];
            const double pi = pst[g] - un * O.hk[2 * (j * B.nx + i) + a];
            lam[side_off(B, sid) + pos] = -O.bB[side_off(B, sid) + pos] * un + pi;
        }
    }
    __syncthreads();
    const double vol = md.h[0] * md.h[1];
    const double* fm = P.f + md.cell_off;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x)
        rt[c] = source_rhs(B, O, fm, nxg, vol, md.h[1], md.h[0], lam, c % B.nx, c / B.nx);
    __syncthreads();
    if (threadIdx.x < 32) {
        RhsStored rs{rt};
        warp_solve<T>(B, O, Sinv, cys, x, mixed ? w : (T*)x, zbuf, rs, Mth.ir_tol, Mth.max_ir, &flags[0]);
    }
    __syncthreads();

    // seeds on Omega_i, taken and cleared (the forward overwrote them)
    for (size_t c = threadIdx.x; c < n; c += blockDim.x) {
        rt[c] = 0.0;
        su[4 * c] = su[4 * c + 1] = su[4 * c + 2] = su[4 * c + 3] = 0.0;
    }
    __syncthreads();
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int offx = sd.lo[0] - B.lo[0], offy = sd.lo[1] - B.lo[1];
    double* gpg = A.gp + md.cell_off;
    double* gug = A.gu + md.cell_off * 4;
    for (int c = threadIdx.x; c < nIx * nIy; c += blockDim.x) {
        const int i = c % nIx + offx, j = c / nIx + offy;
        const int cl = j * B.nx + i;
        const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
        rt[cl] = gpg[g];
        gpg[g] = 0.0;
        for (int s = 0; s < 4; ++s) {
            su[4 * cl + s] = gug[g * 4 + s];
            gug[g * 4 + s] = 0.0;
        }
    }
    __syncthreads();
    // adjoint right-hand side gp + (du/dp)^T gu
    const double rax = 1.0 / md.h[1], ray = 1.0 / md.h[0];
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        const int i = c % B.nx, j = c / B.nx;
        double r = rt[c];
        if (i < B.nx - 1) r += O.cx[c] * (su[4 * c + 1] - su[4 * (c + 1)]) * rax;
        if (i > 0) r -= O.cx[c - 1] * (su[4 * (c - 1) + 1] - su[4 * c]) * rax;
        if (j < B.ny - 1) r += O.cy[c] * (su[4 * c + 3] - su[4 * (c + B.nx) + 2]) * ray;
        if (j > 0) r -= O.cy[c - B.nx] * (su[4 * (c - B.nx) + 3] - su[4 * c + 2]) * ray;
        if (i == 0 && B.kind[0]) r += O.bT[side_off(B, 0) + j] * su[4 * c] * rax;
        if (i == B.nx - 1 && B.kind[1]) r += O.bT[side_off(B, 1) + j] * su[4 * c + 1] * rax;
        if (j == 0 && B.kind[2]) r += O.bT[side_off(B, 2) + i] * su[4 * c + 2] * ray;
        if (j == B.ny - 1 && B.kind[3]) r += O.bT[side_off(B, 3) + i] * su[4 * c + 3] * ray;
        rt[c] = r;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        RhsStored rs{rt};
        warp_solve<T>(B, O, Sinv, cys, mu, mixed ? w : (T*)mu, zbuf, rs, Mth.ir_tol, Mth.max_ir, &flags[0]);
    }
    __syncthreads();

    // interior faces: dL/dTf = (gu_L - gu_R) dp / a - (mu_L - mu_R) dp
    double* gTf = A.gTf + md.cell_off * 3;
    double* ghk = A.ghk + md.cell_off * 3;
    double* gwh = A.gwh + md.cell_off * 3;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        const int i = c % B.nx, j = c / B.nx;
        const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
        if (i < B.nx - 1) {
            const double dp = x[c] - x[c + 1];
            gTf[g * 3] += ((su[4 * c + 1] - su[4 * (c + 1)]) * rax - (mu[c] - mu[c + 1])) * dp;
        }
        if (j < B.ny - 1) {
            const double dp = x[c] - x[c + B.nx];
            gTf[g * 3 + 1] += ((su[4 * c + 3] - su[4 * (c + B.nx) + 2]) * ray - (mu[c] - mu[c + B.nx])) * dp;
        }
    }
    // box sides one at a time (a corner cell lies on two sides)
    for (int sid = 0; sid < 4; ++sid) {
        if (B.kind[sid] != 0) {
            const int a = sid >> 1;
            const int len = a == 0 ? B.ny : B.nx;
            const double rarea = a == 0 ? rax : ray;
            for (int pos = threadIdx.x; pos < len; pos += blockDim.x) {
                int i, j;
                if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; }
                else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; }
                const int c = j * B.nx + i;
                const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
                const double Tb = O.bT[side_off(B, sid) + pos];
                const double sc = su[4 * c + sid] * rarea;
                const double q = -Tb * Tb * rarea;   // dT/d(h/2K); alpha * q = dT/d(H/K_H)
                if (B.kind[sid] == 2) {
                    const double lv = lam[side_off(B, sid) + pos];
                    const double gT = (x[c] - lv) * (sc - mu[c]);
                    const double gl = Tb * (mu[c] - sc);
                    const double un = ust[g * 4 + sid];
                    const long long gf = (sid & 1) ? g : g - (a == 0 ? 1 : nxg);
                    // lambda = -alpha wh u.n + p - u.n hk
                    ghk[g * 3 + a] += gT * q - gl * un;
                    gwh[gf * 3 + a] += B.alpha * (gT * q - gl * un);
                    gpg[g] += gl;
                    gug[g * 4 + sid] += gl * (-O.bB[side_off(B, sid) + pos] - O.hk[2 * c + a]);
                } else {
                    const double gT = (x[c] - B.val[sid]) * (sc - mu[c]);
                    ghk[g * 3 + a] += gT * q;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && flags[0]) atomicOr(&P.status[0], ST_NO_CONV);
}

// ---------------------------------------------------------------------------
// Superposition backwards: p = pbar + sum_k X_k Psi_k on Omega_i, Gamma_i
// velocities ubar + sum_k X_k U_k, interior and Dirichlet faces from p.
// Writes dL/d(assembled pressure) and dL/d(Gamma velocities) per item and
// dL/dX.  One CTA per subdomain (Omega_i are disjoint).
// ---------------------------------------------------------------------------
__global__ void k_adj_assemble2d(DevPtrs P, AdjPtrs A) {
    extern __shared__ double ash[];
    const int item = blockIdx.x;
    const SubDev sd = P.sub[item];
    const MemberDev& md = P.mem[sd.member];
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int n = nIx * nIy;
    double* ps = ash;
    double* gq = ash + P.ncell_i_max;
    const double* xs = A.X + sd.col0;
    const double* Psi = P.Psi + (size_t)item * P.nbasis_max * P.ncell_i_max;
    const double* pb = P.pbar + (size_t)item * P.ncell_i_max;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double v = pb[c];
        for (int k = 0; k < sd.nbasis; ++k) v += xs[k] * Psi[(size_t)k * P.ncell_i_max + c];
        ps[c] = v;
    }
    __syncthreads();
    const int nxg = md.n[0];
    const double* Tf = P.Tf + md.cell_off * 3;
    const double* hk = P.hk + md.cell_off * 3;
    const double* gpg = A.gp + md.cell_off;
    const double* gug = A.gu + md.cell_off * 4;
    double* gTf = A.gTf + md.cell_off * 3;
    double* ghk = A.ghk + md.cell_off * 3;
    double* gugi = A.gug + (size_t)item * MRCM_MAXSIDE * P.side_max;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int i = c % nIx, j = c / nIx;
        const long long g = (sd.lo[0] + i) + (long long)nxg * (sd.lo[1] + j);
        const double pc = ps[c];
        double r = gpg[g];
        for (int sid = 0; sid < 4; ++sid) {
            const int a = sid >> 1;
            const bool hi = sid & 1;
            const int li = a == 0 ? i : j;
            const int lext = a == 0 ? nIx : nIy;
            const bool edge = hi ? (li == lext - 1) : (li == 0);
            const double rarea = a == 0 ? 1.0 / md.h[1] : 1.0 / md.h[0];
            const double guo = gug[g * 4 + sid];
            if (!edge) {
                const int cn = c + (a == 0 ? (hi ? 1 : -1) : (hi ? nIx : -nIx));
                const long long gn = g + (a == 0 ? (hi ? 1 : -1) : (hi ? nxg : -nxg));
                const double T = Tf[(hi ? g : gn) * 3 + a];
                const double dl = guo - gug[gn * 4 + (sid ^ 1)];
                r += T * dl * rarea;
                if (hi) gTf[g * 3 + a] += dl * (pc - ps[cn]) * rarea;
            } else if (sd.side_mask & (1 << sid)) {
                gugi[sid * P.side_max + (a == 0 ? j : i)] = guo;
            } else if (md.bc_kind[sid] == 1) {
                // T = 2 a K / h = a / hk
                const double T = rarea > 0 ? 1.0 / (hk[g * 3 + a] * rarea) : 0.0;
                r += T * guo * rarea;
                ghk[g * 3 + a] += guo * (pc - md.bc_val[sid]) * rarea * (-T * T * rarea);
            }
        }
        gq[c] = r;
        A.gps[(size_t)item * P.ncell_i_max + c] = r;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < sd.nbasis; k += nw) {
        const double* Pk = Psi + (size_t)k * P.ncell_i_max;
        double s = 0.0;
        for (int c = lane; c < n; c += 32) s += gq[c] * Pk[c];
        const double* Ugk = P.Ug + ((size_t)item * P.nbasis_max + k) * MRCM_MAXSIDE * P.side_max;
        for (int sid = 0; sid < 4; ++sid) {
            if (!(sd.side_mask & (1 << sid))) continue;
            const int len = (sid >> 1) == 0 ? nIy : nIx;
            for (int e = lane; e < len; e += 32) s += gugi[sid * P.side_max + e] * Ugk[sid * P.side_max + e];
        }
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) A.gX[sd.col0 + k] = s;
    }
}

// ---------------------------------------------------------------------------
// dL/d(moments) from dL/drhs = y and dL/dG = -y X^T (Eqs. (int_ujump),
// (int_pjump) as assembled by k_if_assemble).  One CTA per subdomain.
// ---------------------------------------------------------------------------
__global__ void k_adj_moments(DevPtrs P, MethodDev Mth, AdjPtrs A) {
    const int s = blockIdx.x;
    const SubDev sd = P.sub[s];
    const MemberDev& md = P.mem[sd.member];
    const int npsi = Mth.npsi, NB = P.nbasis_max;
    const int nslot = sd.nbasis + 1;
    const int total = nslot * MRCM_MAXSIDE * npsi * 2;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int w = t & 1;
        int r = t >> 1;
        const int m = r % npsi;
        r /= npsi;
        const int sid = r % MRCM_MAXSIDE;
        const int slot = r / MRCM_MAXSIDE;
        if (sid >= 2 * md.dim || !(sd.side_mask & (1 << sid))) continue;
        // the row of this moment: flux rows belong to the lower subdomain of
        // the edge (its high side), pressure rows to the upper one (low side)
        const bool own = w == 0 ? (sid & 1) : !(sid & 1);
        const SubDev o = own ? sd : P.sub[sd.nbr[sid]];
        const int q = row_pos(o, md.dim, npsi, w, own ? sid : (sid ^ 1), m);
        if (q < 0) continue;
        const double yv = A.y[o.col0 + q];
        double v;
        const int sl = slot < sd.nbasis ? slot : NB;
        if (slot < sd.nbasis) {
            const double sg = (w == 1 && own) ? -1.0 : 1.0;
            v = -sg * yv * A.X[sd.col0 + slot];
        } else {
            v = w == 0 ? -yv : (own ? yv : -yv);
        }
        A.gmom[((((size_t)s * (NB + 1) + sl) * MRCM_MAXSIDE + sid) * npsi + m) * 2 + w] = v;
    }
}

// ---------------------------------------------------------------------------
// Basis problems (one adjoint solve per basis function on hat-Omega_i) and
// particular problems (one on Omega_i) backwards.  One CTA per job, one
// warp per right-hand side: recompute the forward solution x_k with the
// box factor, form the adjoint right-hand side from dL/d(pressure on
// Omega_i), dL/d(Gamma velocities) and dL/d(moments), solve for mu_k and
// accumulate the face-coefficient adjoints of all k in shared memory; the
// boxes of different jobs overlap, so the totals go out with atomics.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t adj_carve_bytes(int nx, int ny, int nw, bool part) {
    const size_t n = (size_t)nx * ny;
    const size_t per = 2 * (size_t)(nx + ny);
    size_t s = align16(sizeof(double) * n) * 4 + align16(sizeof(double) * 2 * n);   // cd cx cy dsc hk
    s += align16(sizeof(double) * per) * 3;                                           // bT bB gbT
    s += align16(sizeof(T) * sinv_len(nx, ny, sizeof(T))) + align16(sizeof(T) * n) * 2;
    s += align16(sizeof(T) * 64 * nw);
    s += part ? align16(sizeof(double) * n) : 0;
    s += align16(sizeof(double) * n) * 2;                                             // gcx gcy
    s += (align16(sizeof(double) * n) * 3 + (std::is_same<T, float>::value ? align16(sizeof(T) * n) : 0)) * nw;
    return s + 64;
}

template <typename T, int BW>
__global__ void __launch_bounds__(128, 1) k_adj_local2d(DevPtrs P, MethodDev Mth, AdjPtrs A, const Job* jobs) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool mixed = std::is_same<T, float>::value;
    const int nw = blockDim.x >> 5;
    const Job job = jobs[blockIdx.x];
    const SubDev sd = P.sub[job.item];
    const MemberDev& md = P.mem[sd.member];
    const bool basis = job.type == JOB_BASIS;
    __shared__ Box B;
    if (threadIdx.x == 0) {
        if (basis) setup_box(B, md, sd.loh, sd.hih, Mth.alpha_b);
        else setup_box(B, md, sd.lo, sd.hi, Mth.alpha_b);
    }
    __syncthreads();
    const size_t n = (size_t)B.n;
    const int per = 2 * (B.nx + B.ny);
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = smem + o; o += align16(bytes); return p; };
    Ops O;
    O.cd = (double*)take(sizeof(double) * n);
    O.cx = (double*)take(sizeof(double) * n);
    O.cy = (double*)take(sizeof(double) * n);
    O.dsc = (double*)take(sizeof(double) * n);
    O.hk = (double*)take(sizeof(double) * 2 * n);
    O.bT = (double*)take(sizeof(double) * per);
    O.bB = (double*)take(sizeof(double) * per);
    double* gbT = (double*)take(sizeof(double) * per);
    T* Sinv = (T*)take(sizeof(T) * sinv_len(B.nx, B.ny, sizeof(T)));
    T* cys = (T*)take(sizeof(T) * n);
    T* cxs = (T*)take(sizeof(T) * n);
    T* zall = (T*)take(sizeof(T) * 64 * nw);
    double* bsrc = basis ? nullptr : (double*)take(sizeof(double) * n);
    double* gcx = (double*)take(sizeof(double) * n);
    double* gcy = (double*)take(sizeof(double) * n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* x = (double*)take(sizeof(double) * n * nw) + (size_t)warp * n;
    double* mu = (double*)take(sizeof(double) * n * nw) + (size_t)warp * n;
    double* rt = (double*)take(sizeof(double) * n * nw) + (size_t)warp * n;
    T* wv = mixed ? (T*)take(sizeof(T) * n * nw) + (size_t)warp * n : nullptr;
    int* flags = (int*)take(64);
    if (threadIdx.x == 0) { flags[0] = 0; flags[1] = 0; }
    for (size_t c = threadIdx.x; c < n; c += blockDim.x) { gcx[c] = 0.0; gcy[c] = 0.0; }
    for (int t = threadIdx.x; t < per; t += blockDim.x) gbT[t] = 0.0;
    build_ops(B, md, P, O);
    fill_scale(B, O, mixed);
    factor_box<T, BW, false>(B, O, Sinv, cys, cxs, &flags[0]);
    if (flags[0] && threadIdx.x == 0) {
        atomicOr(&P.status[0], ST_NOT_SPD);
        atomicExch(&P.status[2], job.item);
    }

    // with the particular problem on hat-Omega_i (a variant) it is the basis
    // job's last right-hand side, k = nbasis, its vector in the per-box
    // global scratch of the forward pass
    const int nrhs = basis ? sd.nbasis + (Mth.part_hat ? 1 : 0) : 1;
    const int npsi = Mth.npsi;
    const int nxg = md.n[0];
    const double vol = md.h[0] * md.h[1];
    const double ax = md.h[1], ay = md.h[0];
    const double rax = 1.0 / ax, ray = 1.0 / ay;
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int offx = sd.lo[0] - B.lo[0], offy = sd.lo[1] - B.lo[1];
    const double* fm = P.f + md.cell_off;
    double* ghk = A.ghk + md.cell_off * 3;
    double* gwh = A.gwh + md.cell_off * 3;
    double* gTf = A.gTf + md.cell_off * 3;
    const double* gps = A.gps + (size_t)job.item * P.ncell_i_max;
    const double* gugi = A.gug + (size_t)job.item * MRCM_MAXSIDE * P.side_max;
    T* zb = zall + warp * 64;
    for (int k = warp; k < nrhs; k += nw) {
        // forward solution x_k
        int sk = -1, mk = 0;
        const bool pk = !basis || k >= sd.nbasis;   // the particular problem
        if (!pk) {
            int q = k / npsi;
            mk = k % npsi;
            for (int sid = 0; sid < 4; ++sid)
                if (sd.side_mask & (1 << sid)) {
                    if (q == 0) { sk = sid; break; }
                    --q;
                }
            RhsBasis rb{sk, mk};
            warp_solve<T>(B, O, Sinv, cys, x, mixed ? wv : (T*)x, zb, rb, Mth.ir_tol, Mth.max_ir, &flags[1]);
        } else {
            double* bs = basis ? P.bsrc + (size_t)job.item * P.dsc_stride : bsrc;
            for (int c = lane; c < B.n; c += 32)
                bs[c] = source_rhs(B, O, fm, nxg, vol, ax, ay, nullptr, c % B.nx, c / B.nx);
            __syncwarp();
            RhsStored rs{bs};
            warp_solve<T>(B, O, Sinv, cys, x, mixed ? wv : (T*)x, zb, rs, Mth.ir_tol, Mth.max_ir, &flags[1]);
        }
        __syncwarp();
        // adjoint right-hand side
        const double xk = !pk ? A.X[sd.col0 + k] : 1.0;
        const int slot = !pk ? k : P.nbasis_max;
        const double* gm = A.gmom + (((size_t)job.item * (P.nbasis_max + 1) + slot) * MRCM_MAXSIDE) * npsi * 2;
        for (int c = lane; c < B.n; c += 32) rt[c] = 0.0;
        __syncwarp();
        for (int c = lane; c < nIx * nIy; c += 32)
            rt[(c / nIx + offy) * B.nx + (c % nIx + offx)] = xk * gps[c];
        __syncwarp();
        for (int sid = 0; sid < 4; ++sid) {
            if (!(sd.side_mask & (1 << sid))) continue;
            const int a = sid >> 1;
            const int len = a == 0 ? nIy : nIx;
            const double rl = 1.0 / (double)len;
            const double area = a == 0 ? ax : ay;
            const double rarea = a == 0 ? rax : ray;
            for (int e = lane; e < len; e += 32) {
                int i, j;
                if (a == 0) { j = offy + e; i = (sid == 0) ? offx : offx + nIx - 1; }
                else        { i = offx + e; j = (sid == 2) ? offy : offy + nIy - 1; }
                const int cL = j * B.nx + i;
                const long long gL = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
                const double pL = x[cL];
                bool inner;
                int cR, fidx;
                double Tf;
                double* gacc;
                if (sid == 0)      { inner = i > 0;        cR = cL - 1;    fidx = cL - 1;    gacc = gcx; }
                else if (sid == 1) { inner = i < B.nx - 1; cR = cL + 1;    fidx = cL;        gacc = gcx; }
                else if (sid == 2) { inner = j > 0;        cR = cL - B.nx; fidx = cL - B.nx; gacc = gcy; }
                else               { inner = j < B.ny - 1; cR = cL + B.nx; fidx = cL;        gacc = gcy; }
                Tf = inner ? (a == 0 ? O.cx[fidx] : O.cy[fidx]) : 0.0;
                double s0 = 0.0, s1 = 0.0;
                for (int m = 0; m < npsi; ++m) {
                    const double psv = psi_val(m, e, len, rl);
                    s0 += psv * gm[(sid * npsi + m) * 2 + 0];
                    s1 += psv * gm[(sid * npsi + m) * 2 + 1];
                }
                s0 *= area;
                s1 *= area;
                double guo = xk * gugi[sid * P.side_max + e] + s0;
                double uo, lamv = 0.0;
                const int pos = a == 0 ? j : i;
                if (inner) {
                    uo = Tf * (pL - x[cR]) * rarea;
                } else {
                    const int blen = a == 0 ? B.ny : B.nx;
                    if (basis && sid == sk) lamv = psi_val(mk, pos, blen, B.rlen[sid]);
                    uo = O.bT[side_off(B, sid) + pos] * (pL - lamv) * rarea;
                }
                if (basis) {
                    // pressure moment of pi = p - u.n h / (2K)
                    guo -= O.hk[2 * cL + a] * s1;
                    rt[cL] += s1;
                    atomicAdd(&ghk[gL * 3 + a], -uo * s1);
                } else {
                    // pressure moment of beta ubar.n with beta = alpha H / K_H
                    const long long gf = (sid & 1) ? gL : gL - (a == 0 ? 1 : nxg);
                    guo += O.bB[side_off(B, sid) + pos] * s1;
                    atomicAdd(&gwh[gf * 3 + a], B.alpha * uo * s1);
                }
                if (inner) {
                    rt[cL] += Tf * guo * rarea;
                    rt[cR] -= Tf * guo * rarea;
                    atomicAdd(&gacc[fidx], guo * (pL - x[cR]) * rarea);
                } else {
                    const double Tb = O.bT[side_off(B, sid) + pos];
                    rt[cL] += Tb * guo * rarea;
                    atomicAdd(&gbT[side_off(B, sid) + pos], guo * (pL - lamv) * rarea);
                }
            }
            __syncwarp();
        }
        RhsStored rs{rt};
        warp_solve<T>(B, O, Sinv, cys, mu, mixed ? wv : (T*)mu, zb, rs, Mth.ir_tol, Mth.max_ir, &flags[1]);
        __syncwarp();
        // -mu^T (dA/dc) x
        for (int c = lane; c < B.n; c += 32) {
            const int i = c % B.nx, j = c / B.nx;
            if (i < B.nx - 1) atomicAdd(&gcx[c], -(mu[c] - mu[c + 1]) * (x[c] - x[c + 1]));
            if (j < B.ny - 1) atomicAdd(&gcy[c], -(mu[c] - mu[c + B.nx]) * (x[c] - x[c + B.nx]));
        }
        for (int sid = 0; sid < 4; ++sid) {
            if (B.kind[sid] == 0) continue;
            const int a = sid >> 1;
            const int len = a == 0 ? B.ny : B.nx;
            for (int pos = lane; pos < len; pos += 32) {
                int i, j;
                if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; }
                else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; }
                const int c = j * B.nx + i;
                double ref = 0.0;
                if (B.kind[sid] == 2) ref = (basis && sid == sk) ? psi_val(mk, pos, len, B.rlen[sid]) : 0.0;
                else ref = pk ? B.val[sid] : 0.0;
                atomicAdd(&gbT[side_off(B, sid) + pos], -mu[c] * (x[c] - ref));
            }
        }
        __syncwarp();
    }
    __syncthreads();
    // totals of this job -> global face-coefficient adjoints
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        const int i = c % B.nx, j = c / B.nx;
        const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
        if (i < B.nx - 1 && gcx[c] != 0.0) atomicAdd(&gTf[g * 3], gcx[c]);
        if (j < B.ny - 1 && gcy[c] != 0.0) atomicAdd(&gTf[g * 3 + 1], gcy[c]);
    }
    for (int sid = 0; sid < 4; ++sid) {
        if (B.kind[sid] == 0) continue;
        const int a = sid >> 1;
        const int len = a == 0 ? B.ny : B.nx;
        const double rarea = a == 0 ? rax : ray;
        for (int pos = threadIdx.x; pos < len; pos += blockDim.x) {
            int i, j;
            if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; }
            else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; }
            const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
            const double Tb = O.bT[side_off(B, sid) + pos];
            const double v = gbT[side_off(B, sid) + pos] * (-Tb * Tb * rarea);
            if (v == 0.0) continue;
            atomicAdd(&ghk[g * 3 + a], v);
            if (B.kind[sid] == 2) {
                const long long gf = (sid & 1) ? g : g - (a == 0 ? 1 : nxg);
                atomicAdd(&gwh[gf * 3 + a], B.alpha * v);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && flags[1]) atomicOr(&P.status[0], ST_NO_CONV);
}

// ---------------------------------------------------------------------------
// dL/dlog K_c = K_c dL/dK_c from the face-coefficient adjoints:
//   K_L dTf/dK_L = Tf K_R / (K_L + K_R),  K dhk/dK = -hk,
//   K_L dwh/dK_L = -H / (2 K_L)           (wh = H (1/K_L + 1/K_R) / 2).
// ---------------------------------------------------------------------------
__global__ void k_grad_logK(const MemberDev* mem, int nmem, const double* K, const double* Tf,
                            const double* hk, AdjPtrs A, double* out) {
    const int m = blockIdx.y;
    if (m >= nmem) return;
    const MemberDev& md = mem[m];
    const long long nc = (long long)md.n[0] * md.n[1] * md.n[2];
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const long long g = md.cell_off + c;
    const int idx[3] = {(int)(c % md.n[0]), (int)((c / md.n[0]) % md.n[1]),
                        (int)(c / ((long long)md.n[0] * md.n[1]))};
    const long long st[3] = {1, md.n[0], (long long)md.n[0] * md.n[1]};
    const double kc = K[g];
    double s = 0.0;
    for (int a = 0; a < md.dim; ++a) {
        if (idx[a] < md.n[a] - 1) {
            const double kn = K[g + st[a]];
            s += A.gTf[g * 3 + a] * Tf[g * 3 + a] * (kn / (kc + kn));
            s -= A.gwh[g * 3 + a] * md.Hw[a] / (2.0 * kc);
        }
        if (idx[a] > 0) {
            const long long gl = g - st[a];
            const double kl = K[gl];
            s += A.gTf[gl * 3 + a] * Tf[gl * 3 + a] * (kl / (kl + kc));
            s -= A.gwh[gl * 3 + a] * md.Hw[a] / (2.0 * kc);
        }
        s -= A.ghk[g * 3 + a] * hk[g * 3 + a];
    }
    out[g] = s;
}

// K from K or log K (device input), with a positivity check.
__global__ void k_set_K(const double* src, double* K, long long n, int is_log, int* status) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double v = is_log ? exp(src[c]) : src[c];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(&status[0], ST_BAD_K);
    K[c] = v;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t adj_smooth2d_smem(int prec, int nx, int ny) {
    const size_t n = (size_t)nx * ny;
    const size_t per = 2 * (size_t)(nx + ny);
    const size_t tsz = prec == 0 ? sizeof(double) : sizeof(float);
    size_t s = align16(tsz * sinv_len(nx, ny, (int)tsz));
    s += align16(sizeof(double) * n) * 4 + align16(sizeof(double) * 2 * n);
    s += align16(sizeof(double) * per) * 3 + align16(sizeof(double) * n);
    s += align16(tsz * n) + align16(tsz * 64) + align16(sizeof(double) * n) * 2;
    if (prec != 0) s += align16(tsz * n);
    s += align16(sizeof(double) * 4 * n);
    return s + 64;
}

size_t adj_local2d_smem(int prec, int nx, int ny, int nw, bool part) {
    return prec == 0 ? adj_carve_bytes<double>(nx, ny, nw, part) : adj_carve_bytes<float>(nx, ny, nw, part);
}

template <typename K>
static cudaError_t set_smem_attr(K kern, size_t smem, size_t* cur) {
    if (smem > *cur) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        *cur = smem;
    }
    return cudaSuccess;
}

cudaError_t launch_adj_smooth2d(const DevPtrs& P, const MethodDev& M, const AdjPtrs& A, const int* items,
                                int nitems, size_t smem, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    cudaError_t e;
    if (M.prec == 0) {
        static size_t cur = 0;
        if ((e = set_smem_attr(k_adj_smooth2d<double>, smem, &cur)) != cudaSuccess) return e;
        k_adj_smooth2d<double><<<nitems, AS_WARPS * 32, smem, s>>>(P, M, A, items);
    } else {
        static size_t cur = 0;
        if ((e = set_smem_attr(k_adj_smooth2d<float>, smem, &cur)) != cudaSuccess) return e;
        k_adj_smooth2d<float><<<nitems, AS_WARPS * 32, smem, s>>>(P, M, A, items);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_assemble2d(const DevPtrs& P, const AdjPtrs& A, int nitems, int ncell_i_max,
                                  cudaStream_t s) {
    k_adj_assemble2d<<<nitems, 256, sizeof(double) * 2 * ncell_i_max, s>>>(P, A);
    return cudaGetLastError();
}

cudaError_t launch_adj_moments(const DevPtrs& P, const MethodDev& M, const AdjPtrs& A, int nitems,
                               cudaStream_t s) {
    k_adj_moments<<<nitems, 128, 0, s>>>(P, M, A);
    return cudaGetLastError();
}

template <typename T, int BW>
static cudaError_t launch_adj_local_t(const DevPtrs& P, const MethodDev& M, const AdjPtrs& A, const Job* jobs,
                                      int njobs, int nw, size_t smem, cudaStream_t s) {
    static size_t cur = 0;
    cudaError_t e = set_smem_attr(k_adj_local2d<T, BW>, smem, &cur);
    if (e != cudaSuccess) return e;
    k_adj_local2d<T, BW><<<njobs, nw * 32, smem, s>>>(P, M, A, jobs);
    return cudaGetLastError();
}

cudaError_t launch_adj_local2d(const DevPtrs& P, const MethodDev& M, const AdjPtrs& A, const Job* jobs,
                               int njobs, int bw, int nw, size_t smem, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    if (M.prec == 0) {
        if (bw <= 8) return launch_adj_local_t<double, 8>(P, M, A, jobs, njobs, nw, smem, s);
        if (bw <= 16) return launch_adj_local_t<double, 16>(P, M, A, jobs, njobs, nw, smem, s);
        if (bw <= 24) return launch_adj_local_t<double, 24>(P, M, A, jobs, njobs, nw, smem, s);
        return launch_adj_local_t<double, 32>(P, M, A, jobs, njobs, nw, smem, s);
    } else {
        if (bw <= 8) return launch_adj_local_t<float, 8>(P, M, A, jobs, njobs, nw, smem, s);
        if (bw <= 16) return launch_adj_local_t<float, 16>(P, M, A, jobs, njobs, nw, smem, s);
        if (bw <= 24) return launch_adj_local_t<float, 24>(P, M, A, jobs, njobs, nw, smem, s);
        return launch_adj_local_t<float, 32>(P, M, A, jobs, njobs, nw, smem, s);
    }
}

cudaError_t launch_grad_logK(const MemberDev* dmem, int nmem, long long maxcells, const double* K,
                             const double* Tf, const double* hk, const AdjPtrs& A, double* out, cudaStream_t s) {
    dim3 grid((unsigned)((maxcells + 255) / 256), (unsigned)nmem);
    k_grad_logK<<<grid, 256, 0, s>>>(dmem, nmem, K, Tf, hk, A, out);
    return cudaGetLastError();
}

cudaError_t launch_set_K(const double* src, double* K, long long n, int is_log, int* status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_set_K<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, K, n, is_log, status);
    return cudaGetLastError();
}
