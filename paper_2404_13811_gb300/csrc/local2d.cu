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
#include "mrcm_internal.cuh"
#include <type_traits>

namespace {

constexpr int NWARP = 4;

// 1/x in FP64: FP32 reciprocal refined by two Newton steps (error ~ u_64).
__device__ __forceinline__ double rcp64(double x) {
    double r = (double)__frcp_rn((float)x);
    r = r * (2.0 - x * r);
    r = r * (2.0 - x * r);
    return r;
}

// Box description shared by all threads of a CTA.
struct Box {
    int lo[2], hi[2];
    int nx, ny, n;
    int kind[4];      // 0 Neumann, 1 Dirichlet, 2 Robin
    double val[4];    // physical data (g or z)
    double alpha;
    double rlen[4];   // 1 / (faces on the side)
};

// side offsets into the per-side boundary arrays: x sides have ny faces,
// y sides have nx faces.
__device__ __forceinline__ int side_off(const Box& B, int sid) {
    return sid == 0 ? 0 : sid == 1 ? B.ny : sid == 2 ? 2 * B.ny : 2 * B.ny + B.nx;
}

// P0: 1; P1: affine coordinate of the face centre along the side, in [-1, 1].
__device__ __forceinline__ double psi_val(int m, int pos, int len, double rlen) {
    return m == 0 ? 1.0 : (double)(2 * pos + 1 - len) * rlen;
}

// Shared-memory copy of the box operator.
struct Ops {
    double* cd;   // diagonal
    double* cx;   // coupling of cell (i, j) with (i + 1, j)
    double* cy;   // coupling of cell (i, j) with (i, j + 1)
    double* hk;   // h / (2K) per cell, x and y interleaved [2n]
    double* bT;   // boundary-face transmissibility per side
    double* bB;   // Robin beta per side
    double* dsc;  // Jacobi scale (1 in the FP64 form)
};

// Loads the face coefficients of the box and forms the boundary faces.
__device__ void build_ops(const Box& B, const MemberDev& md, const DevPtrs& P, Ops& O) {
    const double* Tf = P.Tf + md.cell_off * 3;
    const double* hkg = P.hk + md.cell_off * 3;
    const double* wh = P.wh + md.cell_off * 3;
    const int nxg = md.n[0];
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        const int i = c % B.nx, j = c / B.nx;
        const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
        O.cx[c] = i < B.nx - 1 ? Tf[g * 3 + 0] : 0.0;
        O.cy[c] = j < B.ny - 1 ? Tf[g * 3 + 1] : 0.0;
        O.hk[2 * c] = hkg[g * 3 + 0];
        O.hk[2 * c + 1] = hkg[g * 3 + 1];
    }
    const double ax = md.h[1], ay = md.h[0];  // face areas (normal to x, normal to y)
    for (int sid = 0; sid < 4; ++sid) {
        const int a = sid >> 1;
        const int len = a == 0 ? B.ny : B.nx;
        const double area = a == 0 ? ax : ay;
        const int off = side_off(B, sid);
        for (int pos = threadIdx.x; pos < len; pos += blockDim.x) {
            int i, j;
            if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; }
            else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; }
            const long long g = (B.lo[0] + i) + (long long)nxg * (B.lo[1] + j);
            const double hin = hkg[g * 3 + a];
            double T = 0.0, beta = 0.0;
            if (B.kind[sid] == 2) {
                // the face to the outside cell: owned by the lower of the two cells
                const long long gf = (sid & 1) ? g : g - (a == 0 ? 1 : nxg);
                beta = B.alpha * wh[gf * 3 + a];
                T = area * rcp64(hin + beta);
            } else if (B.kind[sid] == 1) {
                T = area * rcp64(hin);
            }
            O.bT[off + pos] = T;
            O.bB[off + pos] = beta;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        const int i = c % B.nx, j = c / B.nx;
        double d = O.cx[c] + O.cy[c];
        if (i > 0) d += O.cx[c - 1];
        if (j > 0) d += O.cy[c - B.nx];
        if (i == 0) d += O.bT[side_off(B, 0) + j];
        if (i == B.nx - 1) d += O.bT[side_off(B, 1) + j];
        if (j == 0) d += O.bT[side_off(B, 2) + i];
        if (j == B.ny - 1) d += O.bT[side_off(B, 3) + i];
        O.cd[c] = d;
    }
    __syncthreads();
}

// (A x)_c for the unscaled FP64 operator.
__device__ __forceinline__ double apply_A(const Box& B, const Ops& O, const double* x, int i, int j) {
    const int c = j * B.nx + i;
    double s = O.cd[c] * x[c];
    if (i > 0) s -= O.cx[c - 1] * x[c - 1];
    if (i < B.nx - 1) s -= O.cx[c] * x[c + 1];
    if (j > 0) s -= O.cy[c - B.nx] * x[c - B.nx];
    if (j < B.ny - 1) s -= O.cy[c] * x[c + B.nx];
    return s;
}

// In-register Gauss-Jordan inverse of an SPD b x b block (row i in lane i).
// Pivot reciprocals in FP64.  Writes Sout (row-major, b x b).
template <typename T, int BW>
__device__ void gj_invert(const T* S, T* Sout, int b, T* rowbuf, int* bad) {
    const int lane = threadIdx.x & 31;
    T a[BW];
#pragma unroll
    for (int c = 0; c < BW; ++c) a[c] = (lane < b && c < b) ? S[lane * b + c] : T(lane == c ? 1 : 0);
#pragma unroll
    for (int k = 0; k < BW; ++k) {
        if (k < b) {
            if (lane == k) {
#pragma unroll
                for (int c = 0; c < BW; ++c) rowbuf[c] = a[c];
            }
            __syncwarp();
            double piv = (double)rowbuf[k];
            if (!(piv > 0.0)) {
                if (lane == 0) *bad = 1;
                piv = 1.0;
            }
            // FP32 form: __frcp_rn is the FP64 reciprocal rounded to FP32
            const T ip = std::is_same<T, float>::value ? (T)__frcp_rn((float)piv) : (T)rcp64(piv);
            if (lane == k) {
#pragma unroll
                for (int c = 0; c < BW; ++c) a[c] = (c == k) ? ip : a[c] * ip;
            } else {
                const T fip = a[k] * ip;
#pragma unroll
                for (int c = 0; c < BW; ++c) a[c] = (c == k) ? -fip : a[c] - fip * rowbuf[c];
            }
            __syncwarp();
        }
    }
    if (lane < b) {
#pragma unroll
        for (int c = 0; c < BW; ++c)
            if (c < b) Sout[lane * b + c] = a[c];
    }
    __syncwarp();
}

// Block LDL^T factorisation: Sinv[j] = S_j^{-1}.  cys = scaled line coupling
// (type T).  All threads participate.
template <typename T, int BW>
__device__ void factor_box(const Box& B, const Ops& O, T* Sinv, T* cys, T* Sbuf, T* rowbuf, int* bad) {
    const int b = B.nx, nb = B.ny;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x)
        cys[c] = (T)(O.cy[c] * O.dsc[c] * ((c + b < B.n) ? O.dsc[c + b] : 0.0));
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
            const int i = t / b, k = t - (t / b) * b;
            const int ci = j * b + i, ck = j * b + k;
            if (i == k) {
                double s = O.cd[ci] * O.dsc[ci] * O.dsc[ci];
                if (j > 0) {
                    const double cc = (double)cys[ci - b];
                    s -= cc * cc * (double)Sinv[((j - 1) * b + i) * b + i];
                }
                Sbuf[t] = (T)s;
            } else {
                T s = T(0);
                if (k == i + 1) s = (T)(-O.cx[ci] * O.dsc[ci] * O.dsc[ck]);
                if (k == i - 1) s = (T)(-O.cx[ck] * O.dsc[ci] * O.dsc[ck]);
                if (j > 0) s -= cys[ci - b] * Sinv[((j - 1) * b + i) * b + k] * cys[ck - b];
                Sbuf[t] = s;
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) gj_invert<T, BW>(Sbuf, Sinv + (size_t)j * b * b, b, rowbuf, bad);
        __syncthreads();
    }
}

// One warp sweeps in place: on entry w holds the scaled right-hand side, on
// exit the scaled solution.
template <typename T>
__device__ void warp_sweeps(const T* __restrict__ Sinv, const T* __restrict__ cys, T* w, T* zbuf,
                            int b, int nb) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < nb; ++j) {
        if (lane < b) {
            T z = w[j * b + lane];
            if (j > 0) z += cys[(j - 1) * b + lane] * w[(j - 1) * b + lane];
            zbuf[lane] = z;
        }
        __syncwarp();
        if (lane < b) {
            const T* S = Sinv + (size_t)j * b * b;
            T acc0 = T(0), acc1 = T(0);
            int k = 0;
            for (; k + 1 < b; k += 2) {
                acc0 += S[k * b + lane] * zbuf[k];
                acc1 += S[(k + 1) * b + lane] * zbuf[k + 1];
            }
            if (k < b) acc0 += S[k * b + lane] * zbuf[k];
            w[j * b + lane] = acc0 + acc1;
        }
        __syncwarp();
    }
    for (int j = nb - 2; j >= 0; --j) {
        if (lane < b) zbuf[lane] = cys[j * b + lane] * w[(j + 1) * b + lane];
        __syncwarp();
        if (lane < b) {
            const T* S = Sinv + (size_t)j * b * b;
            T acc0 = T(0), acc1 = T(0);
            int k = 0;
            for (; k + 1 < b; k += 2) {
                acc0 += S[k * b + lane] * zbuf[k];
                acc1 += S[(k + 1) * b + lane] * zbuf[k + 1];
            }
            if (k < b) acc0 += S[k * b + lane] * zbuf[k];
            w[j * b + lane] += acc0 + acc1;
        }
        __syncwarp();
    }
}

// Right-hand side generators -------------------------------------------------

// Basis problem: Robin data psi_m on side sk of the box, homogeneous elsewhere.
struct RhsBasis {
    int sk, m;
    __device__ double operator()(const Box& B, const Ops& O, int i, int j) const {
        const int a = sk >> 1;
        const bool on = (sk == 0 && i == 0) || (sk == 1 && i == B.nx - 1) || (sk == 2 && j == 0) ||
                        (sk == 3 && j == B.ny - 1);
        if (!on) return 0.0;
        const int pos = a == 0 ? j : i;
        const int len = a == 0 ? B.ny : B.nx;
        return O.bT[side_off(B, sk) + pos] * psi_val(m, pos, len, B.rlen[sk]);
    }
};

// Fixed right-hand side kept in shared memory (sources + boundary data).
struct RhsStored {
    const double* b;
    __device__ double operator()(const Box& B, const Ops&, int i, int j) const { return b[j * B.nx + i]; }
};

// f |c| + Dirichlet / Neumann data + Robin data lam (lam may be null).
__device__ double source_rhs(const Box& B, const Ops& O, const double* fm, int nxg, double vol, double ax,
                             double ay, const double* lam, int i, int j) {
    double r = fm[(B.lo[0] + i) + (long long)nxg * (B.lo[1] + j)] * vol;
    const int sides[4] = {i == 0 ? 0 : -1, i == B.nx - 1 ? 1 : -1, j == 0 ? 2 : -1, j == B.ny - 1 ? 3 : -1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int sid = sides[q];
        if (sid < 0) continue;
        const int pos = (sid >> 1) == 0 ? j : i;
        const double area = (sid >> 1) == 0 ? ax : ay;
        if (B.kind[sid] == 1) r += O.bT[side_off(B, sid) + pos] * B.val[sid];
        else if (B.kind[sid] == 0) r -= area * B.val[sid];
        else if (lam) r += O.bT[side_off(B, sid) + pos] * lam[side_off(B, sid) + pos];
    }
    return r;
}

// Solves A x = b for one right-hand side with one warp.  FP64 form: one
// solve.  Mixed form: FP32 sweeps + FP64 residual refinement.  Returns the
// number of sweeps (solves) performed.
template <typename T, typename Rhs>
__device__ int warp_solve(const Box& B, const Ops& O, const T* Sinv, const T* cys, double* x, T* w,
                          T* zbuf, const Rhs& rhs, double tol, int max_ir, int* noconv) {
    const int lane = threadIdx.x & 31;
    const int b = B.nx, nb = B.ny;
    if (std::is_same<T, double>::value) {
        for (int j = 0; j < nb; ++j)
            for (int i = lane; i < b; i += 32) w[j * b + i] = (T)rhs(B, O, i, j);
        __syncwarp();
        warp_sweeps<T>(Sinv, cys, w, zbuf, b, nb);
        return 1;
    } else {
        float bn = 0.f;
        for (int j = 0; j < nb; ++j)
            for (int i = lane; i < b; i += 32) {
                const int c = j * b + i;
                const T wc = (T)(O.dsc[c] * rhs(B, O, i, j));
                x[c] = 0.0;
                w[c] = wc;
                bn = fmaxf(bn, fabsf((float)wc));
            }
        for (int o = 16; o; o >>= 1) bn = fmaxf(bn, __shfl_xor_sync(0xffffffffu, bn, o));
        __syncwarp();
        int it = 0;
        for (; it < max_ir; ++it) {
            warp_sweeps<T>(Sinv, cys, w, zbuf, b, nb);
            for (int c = lane; c < B.n; c += 32) x[c] += O.dsc[c] * (double)w[c];
            __syncwarp();
            // FP64 residual of the unscaled operator; the (scaled) norms are taken in FP32
            float rn = 0.f;
            for (int j = 0; j < nb; ++j)
                for (int i = lane; i < b; i += 32) {
                    const int c = j * b + i;
                    const T wc = (T)(O.dsc[c] * (rhs(B, O, i, j) - apply_A(B, O, x, i, j)));
                    w[c] = wc;
                    rn = fmaxf(rn, fabsf((float)wc));
                }
            for (int o = 16; o; o >>= 1) rn = fmaxf(rn, __shfl_xor_sync(0xffffffffu, rn, o));
            __syncwarp();
            if ((double)rn <= tol * (double)bn || bn == 0.f) { ++it; break; }
            if (it == max_ir - 1 && lane == 0) *noconv = 1;
        }
        return it;
    }
}

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// Shared-memory carve-up ----------------------------------------------------
template <typename T>
struct Carve {
    Ops O;
    T* Sinv;
    T* cys;
    T* Sbuf;
    T* rowbuf;
    T* zbuf;   // NWARP * 32
    double* bsrc; // n: fixed right-hand side of the particular problem
    double* X; // nrhs * n
    T* W;      // nrhs * n
    int* flags;
};

template <typename T>
__host__ __device__ inline size_t carve_bytes(int nx, int ny, int nrhs) {
    const size_t n = (size_t)nx * ny;
    size_t s = align16(sizeof(double) * n) * 4 + align16(sizeof(double) * 2 * n);  // cd cx cy dsc hk
    s += align16(sizeof(double) * 2 * (nx + ny)) * 2;                                 // bT bB
    s += align16(sizeof(T) * n * nx) + align16(sizeof(T) * n) + align16(sizeof(T) * nx * nx);
    s += align16(sizeof(T) * 32) + align16(sizeof(T) * 32 * NWARP) + align16(sizeof(double) * n);
    if (std::is_same<T, float>::value) s += align16(sizeof(double) * n * nrhs);
    s += align16(sizeof(T) * n * nrhs);
    return s + 64;
}

template <typename T>
__device__ Carve<T> carve(unsigned char* base, int nx, int ny, int nrhs) {
    Carve<T> C;
    const size_t n = (size_t)nx * ny;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
    C.O.cd = (double*)take(sizeof(double) * n);
    C.O.cx = (double*)take(sizeof(double) * n);
    C.O.cy = (double*)take(sizeof(double) * n);
    C.O.dsc = (double*)take(sizeof(double) * n);
    C.O.hk = (double*)take(sizeof(double) * 2 * n);
    C.O.bT = (double*)take(sizeof(double) * 2 * (nx + ny));
    C.O.bB = (double*)take(sizeof(double) * 2 * (nx + ny));
    C.Sinv = (T*)take(sizeof(T) * n * nx);
    C.cys = (T*)take(sizeof(T) * n);
    C.Sbuf = (T*)take(sizeof(T) * nx * nx);
    C.rowbuf = (T*)take(sizeof(T) * 32);
    C.zbuf = (T*)take(sizeof(T) * 32 * NWARP);
    C.bsrc = (double*)take(sizeof(double) * n);
    if (std::is_same<T, float>::value) C.X = (double*)take(sizeof(double) * n * nrhs);
    C.W = (T*)take(sizeof(T) * n * nrhs);
    if (std::is_same<T, double>::value) C.X = (double*)C.W;
    C.flags = (int*)take(64);
    return C;
}

__device__ void setup_box(Box& B, const MemberDev& md, const int* lo, const int* hi, double alpha) {
    for (int a = 0; a < 2; ++a) {
        B.lo[a] = lo[a];
        B.hi[a] = hi[a];
    }
    B.nx = hi[0] - lo[0];
    B.ny = hi[1] - lo[1];
    B.n = B.nx * B.ny;
    B.alpha = alpha;
    for (int sid = 0; sid < 4; ++sid) {
        const int a = sid >> 1;
        const bool phys = (sid & 1) ? (hi[a] == md.n[a]) : (lo[a] == 0);
        if (phys) {
            B.kind[sid] = md.bc_kind[sid] == 1 ? 1 : 0;
            B.val[sid] = md.bc_val[sid];
        } else {
            B.kind[sid] = 2;
            B.val[sid] = 0.0;
        }
        B.rlen[sid] = 1.0 / (double)(a == 0 ? B.ny : B.nx);
    }
}

__device__ void fill_scale(const Box& B, Ops& O, bool mixed) {
    for (int c = threadIdx.x; c < B.n; c += blockDim.x)
        O.dsc[c] = mixed ? (double)rsqrtf((float)O.cd[c]) : 1.0;
    __syncthreads();
}

// --- bulk (TMA engine) copy global -> shared with an mbarrier -------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Waits for phase `parity` of the barrier for at most ~2^31 cycles (about a
// second); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Steps 1, 2, 4 and 6 of Algorithm 1 for 2D subdomains.
// ---------------------------------------------------------------------------
template <typename T, int BW>
__global__ void __launch_bounds__(NWARP * 32) k_local2d(DevPtrs P, MethodDev Mth, const Job* jobs) {
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
    const int nrhs = job.type == JOB_BASIS ? sd.nbasis : (job.type == JOB_PART ? 1 : 0);
    Carve<T> C = carve<T>(smem, B.nx, B.ny, nrhs > 0 ? min(nrhs, NWARP) : 1);
    if (threadIdx.x == 0) { C.flags[0] = 0; C.flags[1] = 0; }
    build_ops(B, md, P, C.O);
    fill_scale(B, C.O, mixed);
    factor_box<T, BW>(B, C.O, C.Sinv, C.cys, C.Sbuf, C.rowbuf, &C.flags[0]);

    // keep the factor for the smoothing steps
    const bool keep = (job.type == JOB_SFACT) || (job.type == JOB_BASIS && Mth.same_alpha);
    if (keep) {
        T* dst = (T*)P.fac + (size_t)job.item * P.fac_stride;
        const size_t nS = (size_t)B.n * B.nx;
        for (size_t t = threadIdx.x; t < nS; t += blockDim.x) dst[t] = C.Sinv[t];
        double* dd = P.dsc + (size_t)job.item * P.dsc_stride;
        for (int c = threadIdx.x; c < B.n; c += blockDim.x) dd[c] = C.O.dsc[c];
    }
    if (C.flags[0] && threadIdx.x == 0) {
        atomicOr(&P.status[0], ST_NOT_SPD);
        atomicExch(&P.status[2], job.item);
    }
    if (nrhs == 0) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* zb = C.zbuf + warp * 32;
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
        if (job.type == JOB_BASIS) {
            // k -> (side, m): sides of Gamma_i in increasing id, npsi functions each
            int q = k / npsi;
            mk = k % npsi;
            for (int sid = 0; sid < 4; ++sid)
                if (sd.side_mask & (1 << sid)) {
                    if (q == 0) { sk = sid; break; }
                    --q;
                }
            RhsBasis rb{sk, mk};
            it = warp_solve<T>(B, C.O, C.Sinv, C.cys, x, w, zb, rb, Mth.ir_tol, Mth.max_ir, &C.flags[1]);
        } else {
            // the particular problem: fixed right-hand side staged once
            for (int c = lane; c < B.n; c += 32) {
                const int i = c % B.nx, j = c / B.nx;
                C.bsrc[c] = source_rhs(B, C.O, fm, md.n[0], vol, ax, ay, nullptr, i, j);
            }
            __syncwarp();
            RhsStored rs{C.bsrc};
            it = warp_solve<T>(B, C.O, C.Sinv, C.cys, x, w, zb, rs, Mth.ir_tol, Mth.max_ir, &C.flags[1]);
        }
        maxit = max(maxit, it);
        nsolve += it;
        __syncwarp();
        // ---- outputs: restriction to Omega_i and Gamma_i traces (Eq. (informed_space)) ----
        const int slot = (job.type == JOB_BASIS) ? k : P.nbasis_max;
        double* psi_out = (job.type == JOB_BASIS)
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
            double* ug = (job.type == JOB_BASIS)
                             ? P.Ug + (((size_t)job.item * P.nbasis_max + k) * MRCM_MAXSIDE + sid) * P.side_max
                             : P.ubg + ((size_t)job.item * MRCM_MAXSIDE + sid) * P.side_max;
            double fmv[3] = {0, 0, 0}, pmv[3] = {0, 0, 0};
            for (int e = lane; e < len; e += 32) {
                int i, j;
                if (a == 0) { j = offy + e; i = (sid == 0) ? offx : offx + nIx - 1; }
                else        { i = offx + e; j = (sid == 2) ? offy : offy + nIy - 1; }
                const int cL = j * B.nx + i;
                const double pL = x[cL];
                const double hkL = C.O.hk[2 * cL + a];
                bool inner;
                int cR;
                double Tf;
                if (sid == 0) { inner = i > 0; cR = cL - 1; Tf = inner ? C.O.cx[cL - 1] : 0; }
                else if (sid == 1) { inner = i < B.nx - 1; cR = cL + 1; Tf = inner ? C.O.cx[cL] : 0; }
                else if (sid == 2) { inner = j > 0; cR = cL - B.nx; Tf = inner ? C.O.cy[cL - B.nx] : 0; }
                else { inner = j < B.ny - 1; cR = cL + B.nx; Tf = inner ? C.O.cy[cL] : 0; }
                double uo, pi;
                if (inner) {
                    uo = Tf * (pL - x[cR]) * rarea;
                    pi = pL - uo * hkL;
                } else {
                    // Robin face of the box (l = 0 basis, or the particular problem)
                    const int pos = a == 0 ? j : i;
                    const int blen = a == 0 ? B.ny : B.nx;
                    double lam = 0.0;
                    if (job.type == JOB_BASIS && sid == sk) lam = psi_val(mk, pos, blen, B.rlen[sid]);
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
// coefficients and Robin data are formed; warp 0 runs the sweeps.
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
    if (threadIdx.x == 0) setup_box(B, md, sd.loh, sd.hih, Mth.alpha_s);
    __syncthreads();
    const size_t n = (size_t)B.n;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = smem + o; o += align16(bytes); return p; };
    T* Sinv = (T*)take(sizeof(T) * n * B.nx);
    Ops O;
    O.cd = (double*)take(sizeof(double) * n);
    O.cx = (double*)take(sizeof(double) * n);
    O.cy = (double*)take(sizeof(double) * n);
    O.dsc = (double*)take(sizeof(double) * n);
    O.hk = (double*)take(sizeof(double) * 2 * n);
    O.bT = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    O.bB = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    double* lam = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    double* bsrc = (double*)take(sizeof(double) * n);
    T* cys = (T*)take(sizeof(T) * n);
    T* zbuf = (T*)take(sizeof(T) * 32);
    double* x = (double*)take(sizeof(double) * n);
    T* w = mixed ? (T*)take(sizeof(T) * n) : (T*)x;
    int* flags = (int*)take(64);
    // the bulk copy moves a multiple of 16 bytes; the factor stride and the
    // shared-memory slot are padded to 16 bytes
    const uint32_t sbytes = (uint32_t)((sizeof(T) * n * B.nx + 15) & ~size_t(15));
    const T* Sg = (const T*)P.fac + (size_t)item * P.fac_stride;
    if (threadIdx.x == 0) {
        flags[0] = 0;
        flags[1] = 0;
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, sbytes);
        bulk_g2s(Sinv, Sg, sbytes, &bar);
    }
    build_ops(B, md, P, O);
    const double* dd = P.dsc + (size_t)item * P.dsc_stride;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) O.dsc[c] = dd[c];
    __syncthreads();
    for (int c = threadIdx.x; c < B.n; c += blockDim.x)
        cys[c] = (T)(O.cy[c] * O.dsc[c] * ((c + B.nx < B.n) ? O.dsc[c + B.nx] : 0.0));
    // Robin data from the current solution: lambda = -beta u.n + pi with n the
    // outward normal of hat-Omega_i and pi = p - u.n h / (2K) of the cell inside.
    const double* pst = P.p + md.cell_off;
    const double* ust = P.u + md.cell_off * 4;
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
            const double pi = pst[g] - un * O.hk[2 * (j * B.nx + i) + a];
            lam[side_off(B, sid) + pos] = -O.bB[side_off(B, sid) + pos] * un + pi;
        }
    }
    __syncthreads();
    const double vol = md.h[0] * md.h[1];
    const double* fm = P.f + md.cell_off;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        const int i = c % B.nx, j = c / B.nx;
        bsrc[c] = source_rhs(B, O, fm, md.n[0], vol, md.h[1], md.h[0], lam, i, j);
    }
    __syncthreads();
    int it = 0;
    if (threadIdx.x < 32) {
        const bool ok = mbar_wait(&bar, 0);
        if (!ok) {
            if (threadIdx.x == 0) flags[1] = 1;
        } else {
            RhsStored rs{bsrc};
            it = warp_solve<T>(B, O, Sinv, cys, x, w, zbuf, rs, Mth.ir_tol, Mth.max_ir, &flags[0]);
        }
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
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int offx = sd.lo[0] - B.lo[0], offy = sd.lo[1] - B.lo[1];
    double* pw = P.p + md.cell_off;
    double* uw = P.u + md.cell_off * 4;
    const double rax = 1.0 / md.h[1], ray = 1.0 / md.h[0];
    for (int c = threadIdx.x; c < nIx * nIy; c += blockDim.x) {
        const int i = c % nIx + offx, j = c / nIx + offy;
        const int cl = j * B.nx + i;
        const long long g = (B.lo[0] + i) + (long long)md.n[0] * (B.lo[1] + j);
        const double pc = x[cl];
        pw[g] = pc;
        double uo[4];
        for (int sid = 0; sid < 4; ++sid) {
            const int a = sid >> 1;
            const double rarea = a == 0 ? rax : ray;
            const bool edge = (sid == 0 && i == 0) || (sid == 1 && i == B.nx - 1) || (sid == 2 && j == 0) ||
                              (sid == 3 && j == B.ny - 1);
            if (!edge) {
                const int cn = sid == 0 ? cl - 1 : sid == 1 ? cl + 1 : sid == 2 ? cl - B.nx : cl + B.nx;
                const double Tf = sid == 0 ? O.cx[cl - 1] : sid == 1 ? O.cx[cl] : sid == 2 ? O.cy[cl - B.nx] : O.cy[cl];
                uo[sid] = Tf * (pc - x[cn]) * rarea;
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
size_t local2d_smem(int prec, int nx, int ny, int nrhs) {
    return prec == 0 ? carve_bytes<double>(nx, ny, nrhs) : carve_bytes<float>(nx, ny, nrhs);
}

size_t smooth2d_smem(int prec, int nx, int ny) {
    const size_t n = (size_t)nx * ny;
    const size_t tsz = prec == 0 ? sizeof(double) : sizeof(float);
    size_t s = align16(tsz * n * nx);
    s += align16(sizeof(double) * n) * 4 + align16(sizeof(double) * 2 * n);
    s += align16(sizeof(double) * 2 * (nx + ny)) * 3 + align16(sizeof(double) * n);
    s += align16(tsz * n) + align16(tsz * 32) + align16(sizeof(double) * n);
    if (prec != 0) s += align16(tsz * n);
    return s + 64;
}

template <typename T, int BW>
static cudaError_t launch_local_t(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs,
                                  size_t smem, cudaStream_t s) {
    auto kern = k_local2d<T, BW>;
    static size_t set_smem = 0;
    if (smem > set_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_smem = smem;
    }
    kern<<<njobs, NWARP * 32, smem, s>>>(P, M, jobs);
    return cudaGetLastError();
}

cudaError_t launch_local2d(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs, int bw,
                           size_t smem, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    if (M.prec == 0) {
        if (bw <= 8) return launch_local_t<double, 8>(P, M, jobs, njobs, smem, s);
        if (bw <= 16) return launch_local_t<double, 16>(P, M, jobs, njobs, smem, s);
        if (bw <= 24) return launch_local_t<double, 24>(P, M, jobs, njobs, smem, s);
        return launch_local_t<double, 32>(P, M, jobs, njobs, smem, s);
    } else {
        if (bw <= 8) return launch_local_t<float, 8>(P, M, jobs, njobs, smem, s);
        if (bw <= 16) return launch_local_t<float, 16>(P, M, jobs, njobs, smem, s);
        if (bw <= 24) return launch_local_t<float, 24>(P, M, jobs, njobs, smem, s);
        return launch_local_t<float, 32>(P, M, jobs, njobs, smem, s);
    }
}

cudaError_t launch_smooth2d(const DevPtrs& P, const MethodDev& M, const int* items, int nitems, size_t smem,
                            cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    if (M.prec == 0) {
        auto kern = k_smooth2d<double>;
        static size_t set_smem = 0;
        if (smem > set_smem) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            set_smem = smem;
        }
        kern<<<nitems, SM_WARPS * 32, smem, s>>>(P, M, items);
    } else {
        auto kern = k_smooth2d<float>;
        static size_t set_smem = 0;
        if (smem > set_smem) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            set_smem = smem;
        }
        kern<<<nitems, SM_WARPS * 32, smem, s>>>(P, M, items);
    }
    return cudaGetLastError();
}
