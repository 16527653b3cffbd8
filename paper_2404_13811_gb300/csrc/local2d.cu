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
#include "mrcm_internal.cuh"
#include <type_traits>

namespace {

constexpr int NWARP = 8;

__device__ __forceinline__ double psi_val(int m, int pos, int len) {
    // P0: 1; P1: affine coordinate of the face centre, t in [-1, 1]
    return m == 0 ? 1.0 : (2.0 * (pos + 0.5) / len - 1.0);
}

__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }

// Box description shared by all threads of a CTA.
struct Box {
    int lo[2], hi[2];
    int nx, ny, n;
    int kind[4];      // 0 Neumann, 1 Dirichlet, 2 Robin
    double val[4];    // physical data (g or z)
    double alpha;
};

// side offsets into the per-side boundary arrays: x sides have ny faces,
// y sides have nx faces.
__device__ __forceinline__ int side_off(const Box& B, int sid) {
    return sid == 0 ? 0 : sid == 1 ? B.ny : sid == 2 ? 2 * B.ny : 2 * B.ny + B.nx;
}

// Shared-memory layout of the box operator.
struct Ops {
    double* Kh;   // (nx + 2) * (ny + 2) permeability with a halo ring (0 outside the domain)
    double* cd;   // diagonal
    double* cx;   // coupling of cell (i, j) with (i + 1, j)
    double* cy;   // coupling of cell (i, j) with (i, j + 1)
    double* bT;   // boundary-face transmissibility per side
    double* bB;   // Robin beta per side
    double* dsc;  // Jacobi scale (1 in the FP64 form)
};

// Loads K, builds all face transmissibilities of the box operator.
__device__ void build_ops(const Box& B, const MemberDev& md, const double* __restrict__ K,
                          Ops& O) {
    const int nxh = B.nx + 2;
    const double* Km = K + md.cell_off;
    for (int t = threadIdx.x; t < (B.nx + 2) * (B.ny + 2); t += blockDim.x) {
        int ih = t % nxh, jh = t / nxh;
        int gx = B.lo[0] + ih - 1, gy = B.lo[1] + jh - 1;
        double k = 0.0;
        if (gx >= 0 && gx < md.n[0] && gy >= 0 && gy < md.n[1]) k = Km[gx + (long long)md.n[0] * gy];
        O.Kh[t] = k;
    }
    __syncthreads();
    const double hx = md.h[0], hy = md.h[1];
    const double ax = hy, ay = hx;  // face areas (normal to x, normal to y)
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        int i = c % B.nx, j = c / B.nx;
        double kc = O.Kh[(j + 1) * nxh + i + 1];
        double txp = 0.0, typ = 0.0;
        if (i < B.nx - 1) {
            double kr = O.Kh[(j + 1) * nxh + i + 2];
            txp = ax * 2.0 * kc * kr / (hx * (kc + kr));
        }
        if (j < B.ny - 1) {
            double ku = O.Kh[(j + 2) * nxh + i + 1];
            typ = ay * 2.0 * kc * ku / (hy * (kc + ku));
        }
        O.cx[c] = txp;
        O.cy[c] = typ;
    }
    // boundary faces
    for (int sid = 0; sid < 4; ++sid) {
        const int a = sid >> 1;
        const int len = a == 0 ? B.ny : B.nx;
        const double area = a == 0 ? ax : ay;
        const double h = a == 0 ? hx : hy;
        const int off = side_off(B, sid);
        for (int pos = threadIdx.x; pos < len; pos += blockDim.x) {
            int i, j, io, jo;
            if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; io = (sid == 0) ? i - 1 : i + 1; jo = j; }
            else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; jo = (sid == 2) ? j - 1 : j + 1; io = i; }
            double kin = O.Kh[(j + 1) * nxh + i + 1];
            double T = 0.0, beta = 0.0;
            if (B.kind[sid] == 2) {
                double kout = O.Kh[(jo + 1) * nxh + io + 1];
                beta = B.alpha * md.Hw[a] / harm(kin, kout);
                T = area / (h / (2.0 * kin) + beta);
            } else if (B.kind[sid] == 1) {
                T = 2.0 * area * kin / h;
            }
            O.bT[off + pos] = T;
            O.bB[off + pos] = beta;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        int i = c % B.nx, j = c / B.nx;
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
__device__ __forceinline__ double apply_A(const Box& B, const Ops& O, const double* x, int c) {
    int i = c % B.nx, j = c / B.nx;
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
            const double ipd = 1.0 / piv;
            const T ip = (T)ipd;
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
__device__ void factor_box(const Box& B, const Ops& O, T* Sinv, T* cys, T* Sbuf, T* rowbuf,
                           int* bad) {
    const int b = B.nx, nb = B.ny;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        cys[c] = (T)(O.cy[c] * O.dsc[c] * ((c + b < B.n) ? O.dsc[c + b] : 0.0));
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
            int i = t / b, k = t % b;
            int ci = j * b + i, ck = j * b + k;
            if (i == k) {
                double s = O.cd[ci] * O.dsc[ci] * O.dsc[ci];
                if (j > 0) {
                    double cc = (double)cys[ci - b];
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

// One warp solves (scaled) S-sweeps in place: on entry w holds the scaled
// right-hand side, on exit the scaled solution.
template <typename T>
__device__ void warp_sweeps(const T* __restrict__ Sinv, const T* __restrict__ cys, T* w, T* zbuf,
                            int b, int nb) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < nb; ++j) {
        T z = T(0);
        if (lane < b) {
            z = w[j * b + lane];
            if (j > 0) z += cys[(j - 1) * b + lane] * w[(j - 1) * b + lane];
            zbuf[lane] = z;
        }
        __syncwarp();
        if (lane < b) {
            const T* S = Sinv + (size_t)j * b * b;
            T acc = T(0);
            for (int k = 0; k < b; ++k) acc += S[k * b + lane] * zbuf[k];
            w[j * b + lane] = acc;
        }
        __syncwarp();
    }
    for (int j = nb - 2; j >= 0; --j) {
        if (lane < b) zbuf[lane] = cys[j * b + lane] * w[(j + 1) * b + lane];
        __syncwarp();
        if (lane < b) {
            const T* S = Sinv + (size_t)j * b * b;
            T acc = T(0);
            for (int k = 0; k < b; ++k) acc += S[k * b + lane] * zbuf[k];
            w[j * b + lane] += acc;
        }
        __syncwarp();
    }
}

// Right-hand side generators -------------------------------------------------

// Basis problem k: Robin data psi_m on side sk of the box (homogeneous elsewhere).
struct RhsBasis {
    int sk, m;
    __device__ double operator()(const Box& B, const Ops& O, int c) const {
        int i = c % B.nx, j = c / B.nx;
        int a = sk >> 1;
        bool on = (sk == 0 && i == 0) || (sk == 1 && i == B.nx - 1) || (sk == 2 && j == 0) ||
                  (sk == 3 && j == B.ny - 1);
        if (!on) return 0.0;
        int pos = a == 0 ? j : i;
        int len = a == 0 ? B.ny : B.nx;
        return O.bT[side_off(B, sk) + pos] * psi_val(m, pos, len);
    }
};

// Sources f, g, z plus Robin data lam (may be null = 0).
struct RhsSource {
    const double* f;   // member cell array
    int nxg;           // member grid nx
    double vol, ax, ay;
    const double* lam; // per-side Robin data (side_off layout) or null
    __device__ double operator()(const Box& B, const Ops& O, int c) const {
        int i = c % B.nx, j = c / B.nx;
        double r = f[(B.lo[0] + i) + (long long)nxg * (B.lo[1] + j)] * vol;
        int sides[4] = {i == 0 ? 0 : -1, i == B.nx - 1 ? 1 : -1, j == 0 ? 2 : -1, j == B.ny - 1 ? 3 : -1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int sid = sides[q];
            if (sid < 0) continue;
            int pos = (sid >> 1) == 0 ? j : i;
            double area = (sid >> 1) == 0 ? ax : ay;
            if (B.kind[sid] == 1) r += O.bT[side_off(B, sid) + pos] * B.val[sid];
            else if (B.kind[sid] == 0) r -= area * B.val[sid];
            else if (lam) r += O.bT[side_off(B, sid) + pos] * lam[side_off(B, sid) + pos];
        }
        return r;
    }
};

// Solves A x = b for one right-hand side with one warp.  FP64 form: one
// solve.  Mixed form: FP32 sweeps + FP64 residual refinement.  Returns the
// number of refinement steps.
template <typename T, typename Rhs>
__device__ int warp_solve(const Box& B, const Ops& O, const T* Sinv, const T* cys, double* x,
                          T* w, T* zbuf, const Rhs& rhs, double tol, int max_ir, int* noconv) {
    const int lane = threadIdx.x & 31;
    const int b = B.nx, nb = B.ny, n = B.n;
    if (std::is_same<T, double>::value) {
        // FP64: w aliases x
        for (int c = lane; c < n; c += 32) w[c] = (T)rhs(B, O, c);
        __syncwarp();
        warp_sweeps<T>(Sinv, cys, w, zbuf, b, nb);
        return 1;
    } else {
        double bn = 0.0;
        for (int c = lane; c < n; c += 32) {
            double bc = rhs(B, O, c);
            x[c] = 0.0;
            w[c] = (T)(O.dsc[c] * bc);
            bn = fmax(bn, fabs(bc));
        }
        for (int o = 16; o; o >>= 1) bn = fmax(bn, __shfl_xor_sync(0xffffffffu, bn, o));
        __syncwarp();
        int it = 0;
        for (; it < max_ir; ++it) {
            warp_sweeps<T>(Sinv, cys, w, zbuf, b, nb);
            for (int c = lane; c < n; c += 32) x[c] += O.dsc[c] * (double)w[c];
            __syncwarp();
            double rn = 0.0;
            for (int c = lane; c < n; c += 32) {
                double r = rhs(B, O, c) - apply_A(B, O, x, c);
                rn = fmax(rn, fabs(r));
                w[c] = (T)(O.dsc[c] * r);
            }
            for (int o = 16; o; o >>= 1) rn = fmax(rn, __shfl_xor_sync(0xffffffffu, rn, o));
            __syncwarp();
            if (rn <= tol * bn || bn == 0.0) { ++it; break; }
            if (it == max_ir - 1 && lane == 0) *noconv = 1;
        }
        return it;
    }
}

// Shared-memory carve-up -----------------------------------------------------

template <typename T>
struct Carve {
    Ops O;
    T* Sinv;
    T* cys;
    T* Sbuf;
    T* rowbuf;
    T* zbuf;   // NWARP * 32
    double* X; // nrhs * n
    T* W;      // nrhs * n
    int* flags;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

template <typename T>
__host__ __device__ inline size_t carve_bytes(int nx, int ny, int nrhs) {
    size_t n = (size_t)nx * ny;
    size_t s = 0;
    s += align16(sizeof(double) * (nx + 2) * (ny + 2));
    s += align16(sizeof(double) * n) * 4;               // cd, cx, cy, dsc
    s += align16(sizeof(double) * 2 * (nx + ny)) * 2;   // bT, bB
    s += align16(sizeof(T) * n * nx);                    // Sinv (ny blocks of nx*nx)
    s += align16(sizeof(T) * n);                         // cys
    s += align16(sizeof(T) * nx * nx);                   // Sbuf
    s += align16(sizeof(T) * 32);                        // rowbuf
    s += align16(sizeof(T) * 32 * NWARP);                // zbuf
    if (std::is_same<T, float>::value) s += align16(sizeof(double) * n * nrhs);  // X
    s += align16(sizeof(T) * n * nrhs);                  // W
    s += 64;                                             // flags
    return s;
}

template <typename T>
__device__ Carve<T> carve(unsigned char* base, int nx, int ny, int nrhs) {
    Carve<T> C;
    size_t n = (size_t)nx * ny;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
    C.O.Kh = (double*)take(sizeof(double) * (nx + 2) * (ny + 2));
    C.O.cd = (double*)take(sizeof(double) * n);
    C.O.cx = (double*)take(sizeof(double) * n);
    C.O.cy = (double*)take(sizeof(double) * n);
    C.O.dsc = (double*)take(sizeof(double) * n);
    C.O.bT = (double*)take(sizeof(double) * 2 * (nx + ny));
    C.O.bB = (double*)take(sizeof(double) * 2 * (nx + ny));
    C.Sinv = (T*)take(sizeof(T) * n * nx);
    C.cys = (T*)take(sizeof(T) * n);
    C.Sbuf = (T*)take(sizeof(T) * nx * nx);
    C.rowbuf = (T*)take(sizeof(T) * 32);
    C.zbuf = (T*)take(sizeof(T) * 32 * NWARP);
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
        int a = sid >> 1;
        bool phys = (sid & 1) ? (hi[a] == md.n[a]) : (lo[a] == 0);
        if (phys) {
            B.kind[sid] = md.bc_kind[sid] == 1 ? 1 : 0;
            B.val[sid] = md.bc_val[sid];
        } else {
            B.kind[sid] = 2;
            B.val[sid] = 0.0;
        }
    }
}

__device__ void fill_scale(const Box& B, Ops& O, bool mixed) {
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) O.dsc[c] = mixed ? rsqrt(O.cd[c]) : 1.0;
    __syncthreads();
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
    Carve<T> C = carve<T>(smem, B.nx, B.ny, nrhs > 0 ? nrhs : 1);
    if (threadIdx.x == 0) { C.flags[0] = 0; C.flags[1] = 0; }
    build_ops(B, md, P.K, C.O);
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
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int offx = sd.lo[0] - B.lo[0], offy = sd.lo[1] - B.lo[1];
    int maxit = 0;
    for (int k = warp; k < nrhs; k += NWARP) {
        double* x = C.X + (size_t)k * B.n;
        T* w = C.W + (size_t)k * B.n;
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
            RhsSource rs{P.f + md.cell_off, md.n[0], vol, ax, ay, nullptr};
            it = warp_solve<T>(B, C.O, C.Sinv, C.cys, x, w, zb, rs, Mth.ir_tol, Mth.max_ir, &C.flags[1]);
        }
        maxit = max(maxit, it);
        __syncwarp();
        // ---- outputs: restriction to Omega_i and Gamma_i traces (Eq. (informed_space)) ----
        const int slot = (job.type == JOB_BASIS) ? k : P.nbasis_max;
        double* psi_out = (job.type == JOB_BASIS)
                              ? P.Psi + ((size_t)job.item * P.nbasis_max + k) * P.ncell_i_max
                              : P.pbar + (size_t)job.item * P.ncell_i_max;
        for (int c = lane; c < nIx * nIy; c += 32) {
            int i = c % nIx, j = c / nIx;
            psi_out[c] = x[(j + offy) * B.nx + (i + offx)];
        }
        double* mom = P.mom + (((size_t)job.item * (P.nbasis_max + 1) + slot) * MRCM_MAXSIDE) * npsi * 2;
        for (int sid = 0; sid < 4; ++sid) {
            if (!(sd.side_mask & (1 << sid))) continue;
            const int a = sid >> 1;
            const int len = a == 0 ? nIy : nIx;
            const double area = a == 0 ? ax : ay;
            const double h = md.h[a];
            double* ug = (job.type == JOB_BASIS)
                             ? P.Ug + (((size_t)job.item * P.nbasis_max + k) * MRCM_MAXSIDE + sid) * P.side_max
                             : P.ubg + ((size_t)job.item * MRCM_MAXSIDE + sid) * P.side_max;
            double fm[3] = {0, 0, 0}, pm[3] = {0, 0, 0};
            for (int e = lane; e < len; e += 32) {
                // cell L of Omega_i next to the face, in box coordinates
                int i, j;
                if (a == 0) { j = offy + e; i = (sid == 0) ? offx : offx + nIx - 1; }
                else        { i = offx + e; j = (sid == 2) ? offy : offy + nIy - 1; }
                const int cL = j * B.nx + i;
                const double pL = x[cL];
                const double KL = C.O.Kh[(j + 1) * (B.nx + 2) + i + 1];
                bool inner;
                int cR = -1;
                double Tf;
                if (sid == 0) { inner = i > 0; cR = cL - 1; Tf = inner ? C.O.cx[cL - 1] : 0; }
                else if (sid == 1) { inner = i < B.nx - 1; cR = cL + 1; Tf = inner ? C.O.cx[cL] : 0; }
                else if (sid == 2) { inner = j > 0; cR = cL - B.nx; Tf = inner ? C.O.cy[cL - B.nx] : 0; }
                else { inner = j < B.ny - 1; cR = cL + B.nx; Tf = inner ? C.O.cy[cL] : 0; }
                double uo, pi;
                if (inner) {
                    uo = Tf * (pL - x[cR]) / area;
                    pi = pL - uo * h / (2.0 * KL);
                } else {
                    // Robin face of the box (l = 0 basis, or the particular problem)
                    const int pos = a == 0 ? j : i;
                    const int blen = a == 0 ? B.ny : B.nx;
                    double lam = 0.0;
                    if (job.type == JOB_BASIS && sid == sk) lam = psi_val(mk, pos, blen);
                    uo = C.O.bT[side_off(B, sid) + pos] * (pL - lam) / area;
                    if (job.type == JOB_PART) pi = C.O.bB[side_off(B, sid) + pos] * uo;  // beta ubar.n
                    else pi = pL - uo * h / (2.0 * KL);
                }
                ug[e] = uo;
                for (int m = 0; m < npsi; ++m) {
                    double ps = psi_val(m, e, len);
                    fm[m] += ps * uo * area;
                    pm[m] += area * ps * pi;
                }
            }
            for (int m = 0; m < npsi; ++m) {
                for (int o = 16; o; o >>= 1) {
                    fm[m] += __shfl_xor_sync(0xffffffffu, fm[m], o);
                    pm[m] += __shfl_xor_sync(0xffffffffu, pm[m], o);
                }
                if (lane == 0) {
                    mom[(sid * npsi + m) * 2 + 0] = fm[m];
                    mom[(sid * npsi + m) * 2 + 1] = pm[m];
                }
            }
        }
    }
    if (lane == 0 && maxit > 0) atomicMax(&P.status[1], maxit);
    __syncthreads();
    if (threadIdx.x == 0 && C.flags[1]) atomicOr(&P.status[0], ST_NO_CONV);
}

// ---------------------------------------------------------------------------
// Step 7: one colour phase of a smoothing step (Sec. 3, Eqs. (sm_1)-(sm_2)).
// One warp per subdomain of the colour.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(32) k_smooth2d(DevPtrs P, MethodDev Mth, const int* items) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool mixed = std::is_same<T, float>::value;
    const int item = items[blockIdx.x];
    const SubDev sd = P.sub[item];
    const MemberDev& md = P.mem[sd.member];
    __shared__ Box B;
    if (threadIdx.x == 0) setup_box(B, md, sd.loh, sd.hih, Mth.alpha_s);
    __syncthreads();
    // carve: ops + cys + lam + x + w
    size_t n = (size_t)B.n;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = smem + o; o += align16(bytes); return p; };
    Ops O;
    O.Kh = (double*)take(sizeof(double) * (B.nx + 2) * (B.ny + 2));
    O.cd = (double*)take(sizeof(double) * n);
    O.cx = (double*)take(sizeof(double) * n);
    O.cy = (double*)take(sizeof(double) * n);
    O.dsc = (double*)take(sizeof(double) * n);
    O.bT = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    O.bB = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    double* lam = (double*)take(sizeof(double) * 2 * (B.nx + B.ny));
    T* cys = (T*)take(sizeof(T) * n);
    T* zbuf = (T*)take(sizeof(T) * 32);
    double* x = (double*)take(sizeof(double) * n);
    T* w = mixed ? (T*)take(sizeof(T) * n) : (T*)x;
    int* flags = (int*)take(64);
    if (threadIdx.x == 0) flags[0] = 0;
    build_ops(B, md, P.K, O);
    const double* dd = P.dsc + (size_t)item * P.dsc_stride;
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) O.dsc[c] = dd[c];
    __syncwarp();
    for (int c = threadIdx.x; c < B.n; c += blockDim.x)
        cys[c] = (T)(O.cy[c] * O.dsc[c] * ((c + B.nx < B.n) ? O.dsc[c + B.nx] : 0.0));
    // Robin data from the current solution: lambda = -beta u.n + pi with n the
    // outward normal of hat-Omega_i and pi = p - u.n h / (2K) of the cell inside.
    const int dim = 2;
    const double* pst = P.p + md.cell_off;
    const double* ust = P.u + md.cell_off * 2 * dim;
    for (int sid = 0; sid < 4; ++sid) {
        if (B.kind[sid] != 2) continue;
        const int a = sid >> 1;
        const int len = a == 0 ? B.ny : B.nx;
        for (int pos = threadIdx.x; pos < len; pos += 32) {
            int i, j;
            if (a == 0) { j = pos; i = (sid == 0) ? 0 : B.nx - 1; }
            else        { i = pos; j = (sid == 2) ? 0 : B.ny - 1; }
            long long g = (B.lo[0] + i) + (long long)md.n[0] * (B.lo[1] + j);
            double un = ust[g * 4 + sid];
            double kin = O.Kh[(j + 1) * (B.nx + 2) + i + 1];
            double pi = pst[g] - un * md.h[a] / (2.0 * kin);
            lam[side_off(B, sid) + pos] = -O.bB[side_off(B, sid) + pos] * un + pi;
        }
    }
    __syncwarp();
    const T* Sinv = (const T*)P.fac + (size_t)item * P.fac_stride;
    const double vol = md.h[0] * md.h[1];
    RhsSource rs{P.f + md.cell_off, md.n[0], vol, md.h[1], md.h[0], lam};
    int it = warp_solve<T>(B, O, Sinv, cys, x, w, zbuf, rs, Mth.ir_tol, Mth.max_ir, &flags[0]);
    __syncwarp();
    // overwrite (u, p) on Omega_i with the restriction
    const int nIx = sd.hi[0] - sd.lo[0], nIy = sd.hi[1] - sd.lo[1];
    const int offx = sd.lo[0] - B.lo[0], offy = sd.lo[1] - B.lo[1];
    double* pw = P.p + md.cell_off;
    double* uw = P.u + md.cell_off * 4;
    const double ax = md.h[1], ay = md.h[0];
    for (int c = threadIdx.x; c < nIx * nIy; c += 32) {
        int i = c % nIx + offx, j = c / nIx + offy;
        int cl = j * B.nx + i;
        long long g = (B.lo[0] + i) + (long long)md.n[0] * (B.lo[1] + j);
        double pc = x[cl];
        pw[g] = pc;
        double uo[4];
        for (int sid = 0; sid < 4; ++sid) {
            const int a = sid >> 1;
            const double area = a == 0 ? ax : ay;
            bool edge = (sid == 0 && i == 0) || (sid == 1 && i == B.nx - 1) || (sid == 2 && j == 0) ||
                        (sid == 3 && j == B.ny - 1);
            if (!edge) {
                int cn = sid == 0 ? cl - 1 : sid == 1 ? cl + 1 : sid == 2 ? cl - B.nx : cl + B.nx;
                double Tf = sid == 0 ? O.cx[cl - 1] : sid == 1 ? O.cx[cl] : sid == 2 ? O.cy[cl - B.nx] : O.cy[cl];
                uo[sid] = Tf * (pc - x[cn]) / area;
            } else {
                int pos = a == 0 ? j : i;
                double Tb = O.bT[side_off(B, sid) + pos];
                if (B.kind[sid] == 2) uo[sid] = Tb * (pc - lam[side_off(B, sid) + pos]) / area;
                else if (B.kind[sid] == 1) uo[sid] = Tb * (pc - B.val[sid]) / area;
                else uo[sid] = B.val[sid];
            }
        }
        for (int sid = 0; sid < 4; ++sid) uw[g * 4 + sid] = uo[sid];
    }
    if (threadIdx.x == 0) {
        atomicMax(&P.status[1], it);
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
    size_t n = (size_t)nx * ny;
    size_t s = align16(sizeof(double) * (nx + 2) * (ny + 2)) + align16(sizeof(double) * n) * 4 +
               align16(sizeof(double) * 2 * (nx + ny)) * 3;
    size_t tsz = prec == 0 ? sizeof(double) : sizeof(float);
    s += align16(tsz * n) + align16(tsz * 32) + align16(sizeof(double) * n);
    if (prec != 0) s += align16(tsz * n);
    return s + 64;
}

template <typename T, int BW>
static cudaError_t launch_local_t(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs,
                                  size_t smem, cudaStream_t s) {
    auto kern = k_local2d<T, BW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
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

cudaError_t launch_smooth2d(const DevPtrs& P, const MethodDev& M, const int* items, int nitems,
                            size_t smem, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    if (M.prec == 0) {
        auto kern = k_smooth2d<double>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nitems, 32, smem, s>>>(P, M, items);
    } else {
        auto kern = k_smooth2d<float>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nitems, 32, smem, s>>>(P, M, items);
    }
    return cudaGetLastError();
}
