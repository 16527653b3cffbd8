// Device building blocks of the 2D local solves, shared by the forward
// kernels (local2d.cu) and their adjoints (adjoint2d.cu): the box and its
// cell-centred RT0 operator (Sec. 2.2), the block LDL^T factorisation over
// grid lines, warp-level solves (FP64, or FP32 sweeps with FP64 residual
// refinement), right-hand-side generators and the bulk-copy helpers.
#pragma once
#include "mrcm_internal.cuh"
#include <type_traits>

namespace {

constexpr int NWARP = 4;

// FP32 normal range of an FP64 value, from its exponent bits (integer pipe).
__device__ __forceinline__ bool in_f32_range(double x) {
    const unsigned e11 = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
    return e11 >= 1023u - 126u && e11 <= 1023u + 126u;   // 2^-126 <= |x| < 2^127
}

// 1/x in FP64 by Newton-Raphson iteration for the reciprocal, r <- r (2 - x r),
// from the correctly rounded FP32 reciprocal of x: each step squares the
// relative error (about 2^-23 for the seed, below the FP64 rounding after two
// steps), without the FP64 division.  Outside the FP32 normal range the seed
// would be 0 or infinite, and the FP64 division is used.
__device__ __forceinline__ double rcp64(double x) {
    if (!in_f32_range(x)) return 1.0 / x;
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
        if (O.hk) {   // null where the kernel reads h / 2K from global memory
            O.hk[2 * c] = hkg[g * 3 + 0];
            O.hk[2 * c + 1] = hkg[g * 3 + 1];
        }
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

// --- FP32 <-> FP64 conversions on the integer pipe ---------------------------
// On GB300 every FP64-pipe warp instruction, conversions included, occupies
// the sub-partition's FP64 unit for 64 cycles, and the refinement of the
// mixed form converts twice per cell and step; these do it with integer
// operations instead.  FP32 -> FP64 is exact for normal numbers and zero
// (FP32 subnormals are flushed to zero; infinities and NaN keep their class).
// FP64 -> FP32 truncates the mantissa -- it serves only the right-hand side
// of a correction solve, where an error below one FP32 ulp is immaterial --
// flushes results below the FP32 normal range to zero and takes larger ones
// to infinity (NaN stays NaN).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned hs = u & 0x80000000u;
    const unsigned e11 = e == 0xffu ? 0x7ffu : e + 896u;
    const unsigned hi = e == 0u ? hs : (hs | (e11 << 20) | ((u & 0x7fffffu) >> 3));
    const unsigned lo = e == 0u ? 0u : (u << 29);
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f_bits(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned s = hi & 0x80000000u;
    const int e11 = (int)((hi >> 20) & 0x7ffu);
    const int e = e11 - 896;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned r = s | ((unsigned)e << 23) | m;
    if (e <= 0) r = s;
    if (e >= 255) r = s | 0x7f800000u | ((e11 == 0x7ff && ((hi & 0xfffffu) | lo)) ? 0x400000u : 0u);
    return __uint_as_float(r);
}

// The mixed form refines in Jacobi-scaled variables: O holds D A D (D =
// diag(dsc)) after scale_ops, the iterate is x~ = D^-1 x and the right-hand
// side b~ = D b, so that a residual b~ - (D A D) x~ is five FP64 FMAs per cell
// and an update one FP64 add.  The FP64 form keeps D = I and A.
__device__ void scale_ops(const Box& B, Ops& O) {
    for (int c = threadIdx.x; c < B.n; c += blockDim.x) {
        const int i = c % B.nx, j = c / B.nx;
        const double d = O.dsc[c];
        O.cx[c] = i < B.nx - 1 ? O.cx[c] * d * O.dsc[c + 1] : 0.0;
        O.cy[c] = j < B.ny - 1 ? O.cy[c] * d * O.dsc[c + B.nx] : 0.0;
        O.cd[c] = O.cd[c] * d * d;
    }
    __syncthreads();
}

// b~_c - ((D A D) x~)_c with O scaled.
__device__ __forceinline__ double resid_sc(const Box& B, const Ops& O, const double* x, double bt, int c, int i,
                                           int j) {
    double s = fma(-O.cd[c], x[c], bt);
    if (i > 0) s = fma(O.cx[c - 1], x[c - 1], s);
    if (i < B.nx - 1) s = fma(O.cx[c], x[c + 1], s);
    if (j > 0) s = fma(O.cy[c - B.nx], x[c - B.nx], s);
    if (j < B.ny - 1) s = fma(O.cy[c], x[c + B.nx], s);
    return s;
}

// ---------------------------------------------------------------------------
// Twisted block LDL^T over the grid lines of a box.
//
// The Jacobi-scaled operator is block tridiagonal over its nb lines of b
// cells: diagonal blocks T_j (the couplings inside line j) and off-diagonal
// blocks -C_j, C_j = diag(cys_j), between lines j and j + 1.  It is factored
// from both ends towards the middle line m = nb / 2 (a twisted, or
// burn-at-both-ends, block factorisation):
//   top     S_j = T_j - C_{j-1} S_{j-1}^-1 C_{j-1},                j = 0 .. m - 1
//   bottom  R_j = T_j - C_j R_{j+1}^-1 C_j,                        j = nb - 1 .. m + 1
//   middle  M   = T_m - C_{m-1} S_{m-1}^-1 C_{m-1} - C_m R_{m+1}^-1 C_m
// and S_j^-1 (j < m), M^-1 (j = m), R_j^-1 (j > m) are kept in line order.
// A solve runs two half-length sweeps from the ends, meeting at line m:
//   forward  y_j = S_j^-1 (b_j + C_{j-1} y_{j-1}),  y_j = R_j^-1 (b_j + C_j y_{j+1})
//   middle   x_m = M^-1 (b_m + C_{m-1} y_{m-1} + C_m y_{m+1})
//   back     x_j = y_j + S_j^-1 C_j x_{j+1},        x_j = y_j + R_j^-1 C_{j-1} x_{j-1}
// The blocks are those of a one-sided block LDL^T in another elimination
// order.  The two chains of a solve run interleaved on one warp (a step
// issues both chains' line products, which costs little more than one), so
// a solve is nb / 2 + 1 dependent steps instead of 2 nb - 1; the two chains
// of the factorisation run on two warps (nb / 2 + 1 line inversions in a
// chain instead of nb).
//
// Storage: block j of lines of b cells at j b ld, row-major with row stride
// ld = sld(b).  FP32 rows are read as float4 by one lane each; rows of b
// floats with b / 4 even would put the rows of lanes i and i + 4 (or closer)
// of an 8-lane phase in one bank group, so they are padded by four floats
// (then ld / 4 is odd and the eight rows start in distinct groups).  FP64
// blocks are read by column (no padding).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int sld_of(int b, int tsz) {
    return (tsz == 4 && b % 4 == 0 && (b / 4) % 2 == 0) ? b + 4 : b;
}
template <typename T>
__host__ __device__ constexpr int sld(int b) { return sld_of(b, (int)sizeof(T)); }
__host__ __device__ inline size_t sinv_len(int nx, int ny, int tsz) { return (size_t)ny * nx * sld_of(nx, tsz); }

// In-register Gauss-Jordan inverse of an SPD b x b block (row i in lane i),
// SPD so no pivoting.  The pivot row reaches every lane by shuffles from lane
// k; the pivot lane and the other lanes update with selects (no divergent
// paths), so a step is one chain of b shuffles and b FMAs.  Pivot
// reciprocals: the correctly rounded FP32 reciprocal in the FP32 form, FP64
// otherwise.  EX: b == BW (the width known at compile time).
template <typename T, int BW, bool EX>
__device__ __forceinline__ void gj_regs(T (&a)[BW], int b, int* bad) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < BW; ++k) {
        if (EX || k < b) {
            T rv[BW];
#pragma unroll
            for (int c = 0; c < BW; ++c) rv[c] = __shfl_sync(0xffffffffu, a[c], k);
            T piv = rv[k];
            if (!(piv > T(0))) {
                if (lane == 0) *bad = 1;
                piv = T(1);
            }
            T ip;
            if constexpr (std::is_same<T, float>::value) ip = __frcp_rn(piv);
            else ip = rcp64(piv);
            const bool isk = lane == k;
            const T f = a[k] * ip;
            const T ck = isk ? ip : -f;
            if constexpr (std::is_same<T, float>::value) {
                // FP32 form (Jacobi-scaled, so 0 < piv <= 1 and |1 - ip| <= ip):
                // one FMA per entry and no select -- the other lanes compute
                // a - f rv, the pivot lane, whose row is rv, rv - (1 - ip) rv = ip rv
                const T fl = isk ? T(1) - ip : f;
#pragma unroll
                for (int c = 0; c < BW; ++c) a[c] = (c == k) ? ck : a[c] - fl * rv[c];
            } else {
                // FP64 form (unscaled pivots of any size): the pivot lane computes
                // 0 - (-ip) rv = ip rv, the others a - f rv
                const T fl = isk ? -ip : f;
#pragma unroll
                for (int c = 0; c < BW; ++c) {
                    const T base = isk ? T(0) : a[c];
                    a[c] = (c == k) ? ck : base - fl * rv[c];
                }
            }
        }
    }
}

// Line block j of the twisted factorisation in registers (lane i holds row
// i): T_j minus C S^-1 C for each kept neighbour inverse given (up: the
// inverse of line j - 1, coupled through cys_{j-1}; dn: the inverse of line
// j + 1, coupled through cys_j).  Off-diagonal entries in T, the diagonal
// d_i - sum c_i^2 (S^-1)_ii -- where the cancellation is -- in FP64.  With
// the width known at compile time (EX, FP32) lane i reads row i of the
// (symmetric) neighbour inverse and the coupling vector as float4 and the
// FP64 diagonal converts on the integer pipe (FP32 -> FP64 exact, the FP64
// result truncated to FP32 within one ulp); otherwise lane i reads column i.
template <typename T, int BW, bool EX, bool SC>
__device__ __forceinline__ void form_line(T (&a)[BW], const Ops& O, const T* cys, const T* cxs, int b, int ld,
                                          int j, const T* up, const T* dn) {
    if constexpr (EX) {
        b = BW;
        ld = sld<T>(BW);
    }
    const int i = threadIdx.x & 31;
    const bool act = i < b;
    const int ii = act ? i : 0;
    const int ci = j * b + ii;
    const T cu = up ? cys[ci - b] : T(0);
    const T cn = dn ? cys[ci] : T(0);
    // in-line couplings of cell i: to i + 1 and to i - 1
    const T xr = (act && ii < b - 1) ? cxs[ci] : T(0);
    const T xl = (act && ii > 0) ? cxs[ci - 1] : T(0);
    constexpr bool VEC = EX && std::is_same<T, float>::value && (BW % 4 == 0);
    double d = SC ? O.cd[ci] : O.cd[ci] * O.dsc[ci] * O.dsc[ci];
    if constexpr (VEC) {
        const double cu2 = up ? f2d_bits(cu) * f2d_bits(cu) : 0.0;   // exact in FP64
        const double cn2 = dn ? f2d_bits(cn) * f2d_bits(cn) : 0.0;
        if (up) d = fma(-cu2, f2d_bits(up[ii * ld + ii]), d);
        if (dn) d = fma(-cn2, f2d_bits(dn[ii * ld + ii]), d);
    } else {
        // c (c S_ii), not c^2 S_ii: c^2 leaves the FP64 range for couplings
        // below ~1e-154 (permeabilities scaled that far), c S_ii does not
        if (up) d -= (double)cu * ((double)cu * (double)up[ii * ld + ii]);
        if (dn) d -= (double)cn * ((double)cn * (double)dn[ii * ld + ii]);
    }
    T dT;
    if constexpr (VEC) dT = d2f_bits(d);
    else dT = (T)d;
    if constexpr (VEC) {
        constexpr int NQ = BW / 4;
        float4 ru[NQ], rd[NQ], ku[NQ], kd[NQ];
        if (up) {
            const float4* r = reinterpret_cast<const float4*>(up + ii * ld);
            const float4* k = reinterpret_cast<const float4*>(cys + (j - 1) * b);
#pragma unroll
            for (int q = 0; q < NQ; ++q) { ru[q] = r[q]; ku[q] = k[q]; }
        }
        if (dn) {
            const float4* r = reinterpret_cast<const float4*>(dn + ii * ld);
            const float4* k = reinterpret_cast<const float4*>(cys + j * b);
#pragma unroll
            for (int q = 0; q < NQ; ++q) { rd[q] = r[q]; kd[q] = k[q]; }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float su[4] = {0.f, 0.f, 0.f, 0.f}, sd[4] = {0.f, 0.f, 0.f, 0.f};
            if (up) {
                su[0] = cu * ru[q].x * ku[q].x; su[1] = cu * ru[q].y * ku[q].y;
                su[2] = cu * ru[q].z * ku[q].z; su[3] = cu * ru[q].w * ku[q].w;
            }
            if (dn) {
                sd[0] = cn * rd[q].x * kd[q].x; sd[1] = cn * rd[q].y * kd[q].y;
                sd[2] = cn * rd[q].z * kd[q].z; sd[3] = cn * rd[q].w * kd[q].w;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * q + e;
                const float off = (c == i + 1 ? xr : c == i - 1 ? xl : 0.f) - su[e] - sd[e];
                a[c] = act ? (c == i ? dT : off) : T(i == c ? 1 : 0);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < BW; ++c) {
            T s = T(0);
            if (act && (EX || c < b)) {
                s = c == i + 1 ? xr : c == i - 1 ? xl : T(0);
                // by column (consecutive lanes, consecutive words) where rows are not read as float4
                if (up) s -= cu * up[c * ld + ii] * cys[(j - 1) * b + c];
                if (dn) s -= cn * dn[c * ld + ii] * cys[j * b + c];
            }
            a[c] = (act && (EX || c < b)) ? (c == i ? dT : s) : T(i == c ? 1 : 0);
        }
    }
}

// Stores the inverse held in registers (lane i, entry c) as entry (c, i) of
// the row-major block (consecutive lanes, consecutive words); the inverse of
// an SPD block is symmetric, so this is the block up to rounding.
template <typename T, int BW, bool EX>
__device__ __forceinline__ void store_line(const T (&a)[BW], T* S, int b, int ld) {
    if constexpr (EX) {
        b = BW;
        ld = sld<T>(BW);
    }
    const int i = threadIdx.x & 31;
    if (i < b) {
#pragma unroll
        for (int c = 0; c < BW; ++c)
            if (EX || c < b) S[c * ld + i] = a[c];
    }
}

// Twisted block LDL^T factorisation: Sinv[j] as above.  cys / cxs: the scaled
// line / in-line couplings (type T, formed once by all threads).  Warp 0
// runs the top chain and then the middle line, warp 1 the bottom chain.
// EX: the line width b equals BW.
template <typename T, int BW, bool EX, bool SC = false>
__device__ void factor_box(const Box& B, const Ops& O, T* Sinv, T* cys, T* cxs, int* bad) {
    const int b = EX ? BW : B.nx, nb = B.ny;
    const int ld = sld<T>(b);
    const size_t bl = (size_t)b * ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int c = tid; c < B.n; c += nt) {
        if (SC) {   // the operator is scaled already (scale_ops)
            cys[c] = (T)O.cy[c];
            cxs[c] = (T)(-O.cx[c]);
        } else {
            cys[c] = (T)(O.cy[c] * O.dsc[c] * ((c + b < B.n) ? O.dsc[c + b] : 0.0));
            cxs[c] = (T)(-O.cx[c] * O.dsc[c] * ((c % b) < b - 1 ? O.dsc[c + 1] : 0.0));
        }
    }
    __syncthreads();
    const int warp = tid >> 5;
    const int m = nb >> 1;
    if (warp < 2) {
        const bool top = warp == 0;
        const int cnt = top ? m : nb - 1 - m;
        for (int s = 0; s < cnt; ++s) {
            const int j = top ? s : nb - 1 - s;
            T a[BW];
            form_line<T, BW, EX, SC>(a, O, cys, cxs, b, ld, j, (top && j > 0) ? Sinv + (j - 1) * bl : nullptr,
                                 (!top && j < nb - 1) ? Sinv + (j + 1) * bl : nullptr);
            gj_regs<T, BW, EX>(a, b, bad);
            store_line<T, BW, EX>(a, Sinv + j * bl, b, ld);
            __syncwarp();
        }
    }
    __syncthreads();
    if (warp == 0) {
        T a[BW];
        form_line<T, BW, EX, SC>(a, O, cys, cxs, b, ld, m, m > 0 ? Sinv + (m - 1) * bl : nullptr,
                             m < nb - 1 ? Sinv + (m + 1) * bl : nullptr);
        gj_regs<T, BW, EX>(a, b, bad);
        store_line<T, BW, EX>(a, Sinv + m * bl, b, ld);
    }
    __syncthreads();
}

// --- line products of the sweeps --------------------------------------------
// FP32, line width BB known at compile time (a multiple of 4): lane i holds
// row i of a block as BB / 4 float4, loaded before the line's input is ready;
// the line input is read back as float4 broadcasts; four accumulators.
template <int BB>
struct RowF {
    static constexpr int LD = sld<float>(BB), NQ = BB / 4;
    float4 s[NQ];
    __device__ __forceinline__ void load(const float* __restrict__ S, int lane) {
        const float4* r = reinterpret_cast<const float4*>(S + (lane < BB ? lane : 0) * LD);
#pragma unroll
        for (int q = 0; q < NQ; ++q) s[q] = r[q];
    }
    __device__ __forceinline__ float dot(const float* z) const {
        const float4* z4 = reinterpret_cast<const float4*>(z);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float4 zz = z4[q];
            a0 += s[q].x * zz.x;
            a1 += s[q].y * zz.y;
            a2 += s[q].z * zz.z;
            a3 += s[q].w * zz.w;
        }
        return (a0 + a1) + (a2 + a3);
    }
};

// Any width and type: lane i reads column i by scalar loads (the block is
// symmetric up to rounding), two accumulators.
template <typename T>
__device__ __forceinline__ T dot_col(const T* __restrict__ S, const T* z, int b, int ld, int lane) {
    T a0 = T(0), a1 = T(0);
    if (lane < b) {
        int k = 0;
        for (; k + 1 < b; k += 2) {
            a0 += S[k * ld + lane] * z[k];
            a1 += S[(k + 1) * ld + lane] * z[k + 1];
        }
        if (k < b) a0 += S[k * ld + lane] * z[k];
    }
    return a0 + a1;
}

// Both twisted sweeps by one warp, the two chains interleaved step by step.
// w: the scaled right-hand side in, the scaled solution out (line-major, b
// per line); z: 64 entries (two line inputs), 16-byte aligned.  BB > 0: the
// FP32 row path for lines of BB cells; BB = 0: the column path for any b.
// Steps where both chains have a line run as one unit (both products in one
// loop, so the loads and FMAs of the two chains overlap); the top chain has
// at most one line more than the bottom one, run alone at the end.
template <typename T, int BB>
__device__ void tw_warp(const T* __restrict__ Sinv, const T* __restrict__ cys, T* w, T* z, int b, int nb) {
    if constexpr (BB > 0) b = BB;
    using Row = RowF<(BB > 0 ? BB : 4)>;
    const int ld = BB > 0 ? Row::LD : sld<T>(b);
    const int lane = threadIdx.x & 31;
    const bool act = lane < b;
    const size_t bl = (size_t)b * ld;
    const int m = nb >> 1, ntop = m, nbot = nb - 1 - m;   // ntop - nbot is 0 or 1
    T* zt = z;
    T* zb = z + 32;
    Row Lt, Lb;
    // one line product of each chain (or of the top chain alone)
    auto prod2 = [&](const Row& Rt, const Row& Rb, const T* St, const T* Sb, T& rt, T& rb, bool two) {
        if constexpr (BB > 0) {
            const float4* z4t = reinterpret_cast<const float4*>(zt);
            const float4* z4b = reinterpret_cast<const float4*>(zb);
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
            if (two) {
#pragma unroll
                for (int q = 0; q < Row::NQ; ++q) {
                    const float4 u = z4t[q], v = z4b[q];
                    a0 += Rt.s[q].x * u.x; a1 += Rt.s[q].y * u.y; a2 += Rt.s[q].z * u.z; a3 += Rt.s[q].w * u.w;
                    c0 += Rb.s[q].x * v.x; c1 += Rb.s[q].y * v.y; c2 += Rb.s[q].z * v.z; c3 += Rb.s[q].w * v.w;
                }
                rb = (c0 + c1) + (c2 + c3);
            } else {
#pragma unroll
                for (int q = 0; q < Row::NQ; ++q) {
                    const float4 u = z4t[q];
                    a0 += Rt.s[q].x * u.x; a1 += Rt.s[q].y * u.y; a2 += Rt.s[q].z * u.z; a3 += Rt.s[q].w * u.w;
                }
            }
            rt = (a0 + a1) + (a2 + a3);
        } else {
            rt = dot_col<T>(St, zt, b, ld, lane);
            if (two) rb = dot_col<T>(Sb, zb, b, ld, lane);
        }
    };
    T ct = T(0), cb = T(0);   // this lane's entries of the last finished top / bottom line
    // forward: top j = s, bottom j = nb - 1 - s.  The rows of step s + 1 are
    // loaded at the end of step s (into the other register set), so that
    // their latency overlaps the exchange of the line inputs.
    Row Nt, Nb;
    auto fwd = [&](int s, Row& Ct, Row& Cb, Row& Xt, Row& Xb) {
        const int jt = s, jb = nb - 1 - s;
        if (act) {
            zt[lane] = w[jt * b + lane] + (jt > 0 ? cys[(jt - 1) * b + lane] * ct : T(0));
            zb[lane] = w[jb * b + lane] + (s > 0 ? cys[jb * b + lane] * cb : T(0));
        }
        __syncwarp();
        prod2(Ct, Cb, Sinv + jt * bl, Sinv + jb * bl, ct, cb, true);
        if constexpr (BB > 0) {
            if (s + 1 < nbot) {
                Xt.load((const float*)(Sinv + (jt + 1) * bl), lane);
                Xb.load((const float*)(Sinv + (jb - 1) * bl), lane);
            }
        }
        if (act) {
            w[jt * b + lane] = ct;
            w[jb * b + lane] = cb;
        }
        __syncwarp();
    };
    if constexpr (BB > 0) {
        if (nbot > 0) {
            Nt.load((const float*)Sinv, lane);
            Nb.load((const float*)(Sinv + (nb - 1) * bl), lane);
        }
    }
    {
        Row Pt, Pb;
        int s = 0;
        for (; s + 1 < nbot; s += 2) {
            fwd(s, Nt, Nb, Pt, Pb);
            fwd(s + 1, Pt, Pb, Nt, Nb);
        }
        if (s < nbot) fwd(s, Nt, Nb, Pt, Pb);
    }
    if (ntop > nbot) {   // the last top line, j = ntop - 1
        const int jt = ntop - 1;
        if constexpr (BB > 0) Lt.load((const float*)(Sinv + jt * bl), lane);
        if (act) zt[lane] = w[jt * b + lane] + (jt > 0 ? cys[(jt - 1) * b + lane] * ct : T(0));
        __syncwarp();
        T dummy = T(0);
        prod2(Lt, Lb, Sinv + jt * bl, Sinv, ct, dummy, false);
        if (act) w[jt * b + lane] = ct;
        __syncwarp();
    }
    // middle line
    {
        if constexpr (BB > 0) Lt.load((const float*)(Sinv + m * bl), lane);
        if (act) {
            T zm = w[m * b + lane];
            if (m > 0) zm += cys[(m - 1) * b + lane] * ct;
            if (m < nb - 1) zm += cys[m * b + lane] * cb;
            zt[lane] = zm;
        }
        __syncwarp();
        T dummy = T(0);
        prod2(Lt, Lb, Sinv + m * bl, Sinv, ct, dummy, false);
        cb = ct;
        if (act) w[m * b + lane] = ct;
        __syncwarp();
    }
    // back: top j = m - 1 - s, bottom j = m + 1 + s (rows of the next step
    // prefetched as in the forward sweep)
    auto bwd = [&](int s, Row& Ct, Row& Cb, Row& Xt, Row& Xb) {
        const int jt = m - 1 - s, jb = m + 1 + s;
        T wt = T(0), wb = T(0);
        if (act) {
            zt[lane] = cys[jt * b + lane] * ct;
            zb[lane] = cys[(jb - 1) * b + lane] * cb;
            wt = w[jt * b + lane];
            wb = w[jb * b + lane];
        }
        __syncwarp();
        T pt, pb;
        prod2(Ct, Cb, Sinv + jt * bl, Sinv + jb * bl, pt, pb, true);
        if constexpr (BB > 0) {
            if (s + 1 < nbot) {
                Xt.load((const float*)(Sinv + (jt - 1) * bl), lane);
                Xb.load((const float*)(Sinv + (jb + 1) * bl), lane);
            }
        }
        ct = wt + pt;
        cb = wb + pb;
        if (act) {
            w[jt * b + lane] = ct;
            w[jb * b + lane] = cb;
        }
        __syncwarp();
    };
    {
        Row Pt, Pb;
        if constexpr (BB > 0) {
            if (nbot > 0) {
                Nt.load((const float*)(Sinv + (m - 1) * bl), lane);
                Nb.load((const float*)(Sinv + (m + 1) * bl), lane);
            }
        }
        int s = 0;
        for (; s + 1 < nbot; s += 2) {
            bwd(s, Nt, Nb, Pt, Pb);
            bwd(s + 1, Pt, Pb, Nt, Nb);
        }
        if (s < nbot) bwd(s, Nt, Nb, Pt, Pb);
    }
    if (ntop > nbot) {   // the last top line, j = 0
        if constexpr (BB > 0) Lt.load((const float*)Sinv, lane);
        T wt = T(0);
        if (act) {
            zt[lane] = cys[lane] * ct;
            wt = w[lane];
        }
        __syncwarp();
        T pt, dummy = T(0);
        prod2(Lt, Lb, Sinv, Sinv, pt, dummy, false);
        ct = wt + pt;
        if (act) w[lane] = ct;
        __syncwarp();
    }
}

// Out-of-line entry of one row-path width, for kernels that serve boxes of
// several widths: each width's sweeps get their own register allocation
// (inlined together they would share one and spill).  Called once per
// refinement step.
template <int BB>
__device__ __noinline__ void tw_warp_f32(const float* __restrict__ Sinv, const float* __restrict__ cys, float* w,
                                         float* z, int nb) {
    tw_warp<float, BB>(Sinv, cys, w, z, BB, nb);
}

// Both twisted sweeps on two warps (FP32 row path, lines of BB cells): warp
// 0 runs the top chain (lines 0 .. m - 1) and warp 1 the bottom chain (lines
// nb - 1 .. m + 1), each with its rows prefetched a line ahead; after a
// barrier of the two warps (named barrier 1) warp 0 solves the middle line m
// from both chains' last lines, and after another the two chains run back out
// from it.  The line products of tw_warp in the same order, each chain's
// dependent steps on its own warp; the results agree with tw_warp's to
// rounding (the compiler may fuse the line inputs' multiply-adds
// differently).  Called by threads 0 .. 63; z: 64 entries (one line input per
// warp).
template <int BB>
__device__ void tw_2warp(const float* __restrict__ Sinv, const float* __restrict__ cys, float* w, float* z, int nb) {
    using Row = RowF<BB>;
    constexpr int b = BB;
    const int lane = threadIdx.x & 31, h = (threadIdx.x >> 5) & 1;
    const bool act = lane < b;
    const size_t bl = (size_t)b * Row::LD;
    const int m = nb >> 1;
    const int cnt = h == 0 ? m : nb - 1 - m;   // lines of this warp's chain
    float* zz = z + 32 * h;
    float c = 0.f;   // this lane's entry of the chain's last finished line
    Row N, P;
    auto jf = [&](int s) { return h == 0 ? s : nb - 1 - s; };
    auto fwd = [&](int s, Row& C, Row& X) {
        const int j = jf(s);
        if (act) zz[lane] = w[j * b + lane] + (s > 0 ? cys[(h == 0 ? j - 1 : j) * b + lane] * c : 0.f);
        __syncwarp();
        if (s + 1 < cnt) X.load(Sinv + (size_t)jf(s + 1) * bl, lane);
        c = C.dot(zz);
        if (act) w[j * b + lane] = c;
        __syncwarp();
    };
    if (cnt > 0) N.load(Sinv + (size_t)jf(0) * bl, lane);
    {
        int s = 0;
        for (; s + 1 < cnt; s += 2) {
            fwd(s, N, P);
            fwd(s + 1, P, N);
        }
        if (s < cnt) fwd(s, N, P);
    }
    asm volatile("bar.sync 1, 64;" ::: "memory");
    if (h == 0) {
        Row L;
        L.load(Sinv + (size_t)m * bl, lane);
        if (act) {
            float zm = w[m * b + lane];
            if (m > 0) zm += cys[(m - 1) * b + lane] * w[(m - 1) * b + lane];
            if (m < nb - 1) zm += cys[m * b + lane] * w[(m + 1) * b + lane];
            zz[lane] = zm;
        }
        __syncwarp();
        const float r = L.dot(zz);
        if (act) w[m * b + lane] = r;
    }
    asm volatile("bar.sync 1, 64;" ::: "memory");
    c = act ? w[m * b + lane] : 0.f;
    auto jb = [&](int s) { return h == 0 ? m - 1 - s : m + 1 + s; };
    auto bwd = [&](int s, Row& C, Row& X) {
        const int j = jb(s);
        float wj = 0.f;
        if (act) {
            zz[lane] = cys[(h == 0 ? j : j - 1) * b + lane] * c;
            wj = w[j * b + lane];
        }
        __syncwarp();
        if (s + 1 < cnt) X.load(Sinv + (size_t)jb(s + 1) * bl, lane);
        c = wj + C.dot(zz);
        if (act) w[j * b + lane] = c;
        __syncwarp();
    };
    if (cnt > 0) N.load(Sinv + (size_t)jb(0) * bl, lane);
    {
        int s = 0;
        for (; s + 1 < cnt; s += 2) {
            bwd(s, N, P);
            bwd(s + 1, P, N);
        }
        if (s < cnt) bwd(s, N, P);
    }
}

template <int BB>
__device__ __noinline__ void tw_2warp_f32(const float* __restrict__ Sinv, const float* __restrict__ cys, float* w,
                                          float* z, int nb) {
    tw_2warp<BB>(Sinv, cys, w, z, nb);
}

// The FP32 sweeps of one right-hand side by threads 0 .. 63: two warps on the
// row path of the box's line width where there is one, else warp 0 alone by
// column.  zbuf: 64 entries.  The caller synchronises the block afterwards.
__device__ void warp2_sweeps(const float* __restrict__ Sinv, const float* __restrict__ cys, float* w, float* zbuf,
                             int b, int nb) {
    switch (b) {
        case 8: tw_2warp_f32<8>(Sinv, cys, w, zbuf, nb); return;
        case 12: tw_2warp_f32<12>(Sinv, cys, w, zbuf, nb); return;
        case 16: tw_2warp_f32<16>(Sinv, cys, w, zbuf, nb); return;
        case 20: tw_2warp_f32<20>(Sinv, cys, w, zbuf, nb); return;
        case 24: tw_2warp_f32<24>(Sinv, cys, w, zbuf, nb); return;
        case 28: tw_2warp_f32<28>(Sinv, cys, w, zbuf, nb); return;
        case 32: tw_2warp_f32<32>(Sinv, cys, w, zbuf, nb); return;
        default: break;
    }
    if (threadIdx.x < 32) tw_warp<float, 0>(Sinv, cys, w, zbuf, b, nb);
}

// One warp solves in place (one right-hand side): the twisted sweeps, on the
// FP32 row path of the box's line width where there is one, else by column.
// zbuf: 64 entries of this warp.
template <typename T>
__device__ void warp_sweeps(const T* __restrict__ Sinv, const T* __restrict__ cys, T* w, T* zbuf, int b, int nb) {
    if constexpr (std::is_same<T, float>::value) {
        switch (b) {
            case 8: tw_warp_f32<8>(Sinv, cys, w, zbuf, nb); return;
            case 12: tw_warp_f32<12>(Sinv, cys, w, zbuf, nb); return;
            case 16: tw_warp_f32<16>(Sinv, cys, w, zbuf, nb); return;
            case 20: tw_warp_f32<20>(Sinv, cys, w, zbuf, nb); return;
            case 24: tw_warp_f32<24>(Sinv, cys, w, zbuf, nb); return;
            case 28: tw_warp_f32<28>(Sinv, cys, w, zbuf, nb); return;
            case 32: tw_warp_f32<32>(Sinv, cys, w, zbuf, nb); return;
            default: break;
        }
    }
    tw_warp<T, 0>(Sinv, cys, w, zbuf, b, nb);
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
template <typename T, typename Rhs, int SW = 0>
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
            if constexpr (SW > 0) tw_warp<float, SW>(Sinv, cys, w, zbuf, b, nb);
            else warp_sweeps<T>(Sinv, cys, w, zbuf, b, nb);
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

// One line product of an FP64 CTA-wide sweep: lane's entry of S zin with the
// columns split over the warps (warp q reduces columns [q kq, (q + 1) kq)),
// partial sums met in red (double-buffered by line parity: one block
// barrier per line).  Every warp forms the line input in its own 32 entries
// of zw and returns the full sum.
template <typename T>
__device__ __forceinline__ T cta_line(const T* __restrict__ S, T zin, T* zw, T* red, int& par, int b, int ld) {
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5, nq = blockDim.x >> 5;
    const int kq = (b + nq - 1) / nq, ka = wq * kq, kb = min(b, ka + kq);
    T* z = zw + wq * 32;
    if (lane < b) z[lane] = zin;
    __syncwarp();
    if (lane < b) {
        T acc = T(0);
        for (int k = ka; k < kb; ++k) acc += S[k * ld + lane] * z[k];
        red[(par * nq + wq) * 32 + lane] = acc;
    }
    __syncthreads();
    T s = T(0);
    if (lane < b)
        for (int q = 0; q < nq; ++q) s += red[(par * nq + q) * 32 + lane];
    par ^= 1;
    __syncwarp();
    return s;
}

// The twisted sweeps of a CTA-wide solve.  FP32: warp 0 runs both chains
// interleaved (as in a warp solve); the other warps wait at the closing
// barrier.  FP64 (bound by the narrow FP64 pipe, which every warp's share of
// a line product feeds): one chain after the other with each line product
// split over all warps.  w: the scaled right-hand side in, the solution out;
// zw: 32 entries per warp (at least 64).
template <typename T>
__device__ void cta_sweeps(const T* __restrict__ Sinv, const T* __restrict__ cys, T* w, T* zw, T* red, int b,
                           int nb) {
    if constexpr (std::is_same<T, float>::value) {
        if (threadIdx.x < 32) warp_sweeps<float>(Sinv, cys, w, zw, b, nb);
        __syncthreads();
        return;
    } else {
        const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
        const int ld = sld<T>(b);
        const size_t bl = (size_t)b * ld;
        const int m = nb >> 1;
        int par = 0;
        T cur = T(0);
        for (int j = 0; j < m; ++j) {
            const T zin = lane < b ? w[j * b + lane] + (j > 0 ? cys[(j - 1) * b + lane] * cur : T(0)) : T(0);
            cur = cta_line<T>(Sinv + j * bl, zin, zw, red, par, b, ld);
            if (wq == 0 && lane < b) w[j * b + lane] = cur;
        }
        const T ct = cur;
        cur = T(0);
        for (int j = nb - 1; j > m; --j) {
            const T zin = lane < b ? w[j * b + lane] + (j < nb - 1 ? cys[j * b + lane] * cur : T(0)) : T(0);
            cur = cta_line<T>(Sinv + j * bl, zin, zw, red, par, b, ld);
            if (wq == 0 && lane < b) w[j * b + lane] = cur;
        }
        const T cbt = cur;
        T zm = T(0);
        if (lane < b) {
            zm = w[m * b + lane];
            if (m > 0) zm += cys[(m - 1) * b + lane] * ct;
            if (m < nb - 1) zm += cys[m * b + lane] * cbt;
        }
        const T xm = cta_line<T>(Sinv + m * bl, zm, zw, red, par, b, ld);
        if (wq == 0 && lane < b) w[m * b + lane] = xm;
        cur = xm;
        for (int j = m - 1; j >= 0; --j) {
            const T wf = lane < b ? w[j * b + lane] : T(0);
            const T zin = lane < b ? cys[j * b + lane] * cur : T(0);
            cur = wf + cta_line<T>(Sinv + j * bl, zin, zw, red, par, b, ld);
            if (wq == 0 && lane < b) w[j * b + lane] = cur;
        }
        cur = xm;
        for (int j = m + 1; j < nb; ++j) {
            const T wf = lane < b ? w[j * b + lane] : T(0);
            const T zin = lane < b ? cys[(j - 1) * b + lane] * cur : T(0);
            cur = wf + cta_line<T>(Sinv + j * bl, zin, zw, red, par, b, ld);
            if (wq == 0 && lane < b) w[j * b + lane] = cur;
        }
        __syncthreads();
    }
}

// One right-hand side solved by the whole CTA (as warp_solve: FP64 form one
// solve; mixed form FP32 sweeps + FP64 residual refinement, residual and
// norms over all threads).  nrm: 2 unsigned ints of shared memory.  warm
// (mixed form): x holds a starting iterate on entry and the refinement
// starts from its residual; the stopping rule stays relative to the
// right-hand side, so the result meets the same tolerance, and no sweep is
// run when the start already does.
template <typename T, typename Rhs>
__device__ int cta_solve(const Box& B, const Ops& O, const T* Sinv, const T* cys, double* x, T* w, T* zw, T* red,
                         unsigned int* nrm, const Rhs& rhs, double tol, int max_ir, int* noconv, bool warm = false) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = B.nx, nb = B.ny;
    if (std::is_same<T, double>::value) {
        for (int c = tid; c < B.n; c += nt) w[c] = (T)rhs(B, O, c % b, c / b);
        __syncthreads();
        cta_sweeps<T>(Sinv, cys, w, zw, red, b, nb);
        return 1;
    }
    if (tid < 2) nrm[tid] = 0u;
    __syncthreads();
    float bn = 0.f, r0 = 0.f;
    for (int c = tid; c < B.n; c += nt) {
        const int i = c % b, j = c / b;
        const double bc = rhs(B, O, i, j);
        const T wc = (T)(O.dsc[c] * (warm ? bc - apply_A(B, O, x, i, j) : bc));
        w[c] = wc;
        bn = fmaxf(bn, fabsf((float)(O.dsc[c] * bc)));
        r0 = fmaxf(r0, fabsf((float)wc));
    }
    if (!warm)
        for (int c = tid; c < B.n; c += nt) x[c] = 0.0;
    for (int o = 16; o; o >>= 1) {
        bn = fmaxf(bn, __shfl_xor_sync(0xffffffffu, bn, o));
        r0 = fmaxf(r0, __shfl_xor_sync(0xffffffffu, r0, o));
    }
    if ((tid & 31) == 0) {
        atomicMax(&nrm[0], __float_as_uint(bn));
        atomicMax(&nrm[1], __float_as_uint(r0));
    }
    __syncthreads();
    bn = __uint_as_float(nrm[0]);
    r0 = __uint_as_float(nrm[1]);
    __syncthreads();   // nrm[1] is reset at the top of the first step
    int it = 0;
    if (warm && ((double)r0 <= tol * (double)bn || bn == 0.f)) return 0;
    for (; it < max_ir; ++it) {
        cta_sweeps<T>(Sinv, cys, w, zw, red, b, nb);
        for (int c = tid; c < B.n; c += nt) x[c] += O.dsc[c] * (double)w[c];
        if (tid == 0) nrm[1] = 0u;
        __syncthreads();
        float rn = 0.f;
        for (int c = tid; c < B.n; c += nt) {
            const int i = c % b, j = c / b;
            const T wc = (T)(O.dsc[c] * (rhs(B, O, i, j) - apply_A(B, O, x, i, j)));
            w[c] = wc;
            rn = fmaxf(rn, fabsf((float)wc));
        }
        for (int o = 16; o; o >>= 1) rn = fmaxf(rn, __shfl_xor_sync(0xffffffffu, rn, o));
        if ((tid & 31) == 0) atomicMax(&nrm[1], __float_as_uint(rn));
        __syncthreads();
        rn = __uint_as_float(nrm[1]);
        if ((double)rn <= tol * (double)bn || bn == 0.f) { ++it; break; }
        if (it == max_ir - 1 && tid == 0) *noconv = 1;
        __syncthreads();   // nrm[1] is reset at the top of the next step
    }
    __syncthreads();
    return it;
}

// --- the mixed form's refinement in scaled variables -------------------------
// Right-hand sides b~ for the scaled solves.  Basis problem: nonzero only on
// the Robin side sk, where lane pos holds b~ of the side's face pos (a
// register, fetched by shuffle: every lane of the warp calls it); stored:
// an array of b~.
struct RhsScSide {
    int sk;
    double mine;   // b~ of face `lane` of side sk (0 beyond the side)
    __device__ double operator()(const Box& B, int i, int j) const {
        const bool on = (sk == 0 && i == 0) || (sk == 1 && i == B.nx - 1) || (sk == 2 && j == 0) ||
                        (sk == 3 && j == B.ny - 1);
        const double v = __shfl_sync(0xffffffffu, mine, (sk >> 1) == 0 ? j : i);
        return on ? v : 0.0;
    }
};
struct RhsScStored {
    const double* b;
    __device__ double operator()(const Box& B, int i, int j) const { return b[j * B.nx + i]; }
};

// (i, j) of cell c; the line width is a compile-time constant when SW > 0.
template <int SW>
__device__ __forceinline__ void cell_ij(int c, int b, int& i, int& j) {
    if constexpr (SW > 0) {
        i = c % SW;
        j = c / SW;
    } else {
        i = c % b;
        j = c / b;
    }
}

// One right-hand side by one warp in the mixed form: FP32 twisted sweeps of
// the kept factor, FP64 residuals of the scaled operator, until
// |r~|_inf <= tol |b~|_inf (the stopping rule of warp_solve, in the same
// scaled norm).  Cells are visited 32 at a time by all lanes.  On exit x
// holds x~ (the caller scales back with dsc).  Returns the number of sweeps.
template <typename Rhs, int SW = 0>
__device__ int warp_solve_sc(const Box& B, const Ops& O, const float* Sinv, const float* cys, double* x, float* w,
                             float* zbuf, const Rhs& rhs, double tol, int max_ir, int* noconv) {
    const int lane = threadIdx.x & 31;
    const int b = B.nx, nb = B.ny;
    const int nit = (B.n + 31) >> 5;
    float bn = 0.f;
    for (int k = 0; k < nit; ++k) {
        const int c = k * 32 + lane;
        const bool ok = c < B.n;
        int i, j;
        cell_ij<SW>(ok ? c : 0, b, i, j);
        const double bt = rhs(B, i, j);
        if (ok) {
            const float wc = d2f_bits(bt);
            x[c] = 0.0;
            w[c] = wc;
            bn = fmaxf(bn, fabsf(wc));
        }
    }
    for (int o = 16; o; o >>= 1) bn = fmaxf(bn, __shfl_xor_sync(0xffffffffu, bn, o));
    __syncwarp();
    int it = 0;
    for (; it < max_ir; ++it) {
        if constexpr (SW > 0) tw_warp<float, SW>(Sinv, cys, w, zbuf, b, nb);
        else warp_sweeps<float>(Sinv, cys, w, zbuf, b, nb);
        for (int c = lane; c < B.n; c += 32) x[c] += f2d_bits(w[c]);
        __syncwarp();
        float rn = 0.f;
        for (int k = 0; k < nit; ++k) {
            const int c = k * 32 + lane;
            const bool ok = c < B.n;
            int i, j;
            cell_ij<SW>(ok ? c : 0, b, i, j);
            const double bt = rhs(B, i, j);
            if (ok) {
                const float wc = d2f_bits(resid_sc(B, O, x, bt, c, i, j));
                w[c] = wc;
                rn = fmaxf(rn, fabsf(wc));
            }
        }
        for (int o = 16; o; o >>= 1) rn = fmaxf(rn, __shfl_xor_sync(0xffffffffu, rn, o));
        __syncwarp();
        if ((double)rn <= tol * (double)bn || bn == 0.f) { ++it; break; }
        if (it == max_ir - 1 && lane == 0) *noconv = 1;
    }
    return it;
}

// The same by the whole CTA (the smoothing solves): sweeps by warp 0 (both
// chains), FP64 updates and residuals over all threads.  warm: x holds a
// starting x~ and the refinement starts from its residual (stopping rule
// still relative to b~; no sweep when the start meets it).  b~ is stored.
__device__ int cta_solve_sc(const Box& B, const Ops& O, const float* Sinv, const float* cys, double* x, float* w,
                            float* zw, unsigned int* nrm, const double* bt, double tol, int max_ir, int* noconv,
                            bool warm) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = B.nx, nb = B.ny;
    if (tid < 2) nrm[tid] = 0u;
    __syncthreads();
    float bn = 0.f, r0 = 0.f;
    for (int c = tid; c < B.n; c += nt) {
        const int i = c % b, j = c / b;
        const float wb = d2f_bits(bt[c]);
        const float wc = warm ? d2f_bits(resid_sc(B, O, x, bt[c], c, i, j)) : wb;
        w[c] = wc;
        bn = fmaxf(bn, fabsf(wb));
        r0 = fmaxf(r0, fabsf(wc));
    }
    if (!warm)
        for (int c = tid; c < B.n; c += nt) x[c] = 0.0;
    for (int o = 16; o; o >>= 1) {
        bn = fmaxf(bn, __shfl_xor_sync(0xffffffffu, bn, o));
        r0 = fmaxf(r0, __shfl_xor_sync(0xffffffffu, r0, o));
    }
    if ((tid & 31) == 0) {
        atomicMax(&nrm[0], __float_as_uint(bn));
        atomicMax(&nrm[1], __float_as_uint(r0));
    }
    __syncthreads();
    bn = __uint_as_float(nrm[0]);
    r0 = __uint_as_float(nrm[1]);
    __syncthreads();   // nrm[1] is reset at the top of the first step
    int it = 0;
    if (warm && ((double)r0 <= tol * (double)bn || bn == 0.f)) return 0;
    for (; it < max_ir; ++it) {
        if (tid < 64) warp2_sweeps(Sinv, cys, w, zw, b, nb);
        __syncthreads();
        for (int c = tid; c < B.n; c += nt) x[c] += f2d_bits(w[c]);
        if (tid == 0) nrm[1] = 0u;
        __syncthreads();
        float rn = 0.f;
        for (int c = tid; c < B.n; c += nt) {
            const int i = c % b, j = c / b;
            const float wc = d2f_bits(resid_sc(B, O, x, bt[c], c, i, j));
            w[c] = wc;
            rn = fmaxf(rn, fabsf(wc));
        }
        for (int o = 16; o; o >>= 1) rn = fmaxf(rn, __shfl_xor_sync(0xffffffffu, rn, o));
        if ((tid & 31) == 0) atomicMax(&nrm[1], __float_as_uint(rn));
        __syncthreads();
        rn = __uint_as_float(nrm[1]);
        if ((double)rn <= tol * (double)bn || bn == 0.f) { ++it; break; }
        if (it == max_ir - 1 && tid == 0) *noconv = 1;
        __syncthreads();   // nrm[1] is reset at the top of the next step
    }
    __syncthreads();
    return it;
}

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// The smoothing pack of one 2D subdomain: everything the smoothing solves
// need that does not change between smoothing steps, written once after the
// factorisation in the byte layout the smoothing kernel's shared memory
// starts with, so that one bulk copy stages it.  S^-1 blocks first (the
// factor slot other kernels read), then the FP64 operator (diagonal, x / y
// couplings, Jacobi scaling), the box-side transmissibilities and Robin
// beta, the fixed part of the right-hand side (sources and physical
// boundary data) and the scaled y couplings of the sweeps.  Every field
// starts on 16 bytes; the total is a multiple of 16.
struct SPack {
    size_t cd, cx, cy, dsc, bT, bB, bst, cys, bytes;
};

__host__ __device__ inline SPack spack_layout(int nx, int ny, size_t tsz) {
    SPack L;
    const size_t n = (size_t)nx * ny, m = 2 * (size_t)(nx + ny);
    size_t o = align16(tsz * sinv_len(nx, ny, (int)tsz));
    L.cd = o;  o += align16(sizeof(double) * n);
    L.cx = o;  o += align16(sizeof(double) * n);
    L.cy = o;  o += align16(sizeof(double) * n);
    L.dsc = o; o += align16(sizeof(double) * n);
    L.bT = o;  o += align16(sizeof(double) * m);
    L.bB = o;  o += align16(sizeof(double) * m);
    L.bst = o; o += align16(sizeof(double) * n);
    L.cys = o; o += align16(tsz * n);
    L.bytes = o;
    return L;
}

// Shared-memory carve-up ----------------------------------------------------
template <typename T>
struct Carve {
    Ops O;
    T* Sinv;
    T* cys;
    T* cxs;
    T* zbuf;   // NWARP * 64: two line inputs per warp
    double* bsrc; // n: fixed right-hand side of the particular problem
    double* X; // nrhs * n
    T* W;      // nrhs * n
    int* flags;
    size_t end;   // bytes of shared memory the layout takes
};

template <typename T>
// (the basis / particular kernel keeps no h / 2K array -- it reads the few
// values it needs at the Gamma faces from global memory -- and a stored
// right-hand side only for the particular problem, so that two CTAs of the
// 24 x 24 basis boxes fit on one SM)
__host__ __device__ inline size_t carve_bytes(int nx, int ny, int nrhs, bool part) {
    const size_t n = (size_t)nx * ny;
    size_t s = align16(sizeof(double) * n) * 4;                                      // cd cx cy dsc
    s += align16(sizeof(double) * 2 * (nx + ny)) * 2;                                 // bT bB
    s += align16(sizeof(T) * sinv_len(nx, ny, sizeof(T))) + align16(sizeof(T) * n);   // Sinv, cys (cxs lives in W)
    s += align16(sizeof(T) * 64 * NWARP) + (part ? align16(sizeof(double) * n) : 0);
    if (std::is_same<T, float>::value) s += align16(sizeof(double) * n * nrhs);
    s += align16(sizeof(T) * n * nrhs);
    return s + 64;
}

template <typename T>
__device__ Carve<T> carve(unsigned char* base, int nx, int ny, int nrhs, bool part) {
    Carve<T> C;
    const size_t n = (size_t)nx * ny;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
    C.O.cd = (double*)take(sizeof(double) * n);
    C.O.cx = (double*)take(sizeof(double) * n);
    C.O.cy = (double*)take(sizeof(double) * n);
    C.O.dsc = (double*)take(sizeof(double) * n);
    C.O.hk = nullptr;
    C.O.bT = (double*)take(sizeof(double) * 2 * (nx + ny));
    C.O.bB = (double*)take(sizeof(double) * 2 * (nx + ny));
    C.Sinv = (T*)take(sizeof(T) * sinv_len(nx, ny, sizeof(T)));
    C.cys = (T*)take(sizeof(T) * n);
    C.zbuf = (T*)take(sizeof(T) * 64 * NWARP);
    C.bsrc = part ? (double*)take(sizeof(double) * n) : nullptr;
    if (std::is_same<T, float>::value) C.X = (double*)take(sizeof(double) * n * nrhs);
    C.W = (T*)take(sizeof(T) * n * nrhs);
    if (std::is_same<T, double>::value) C.X = (double*)C.W;
    C.cxs = C.W;   // the in-line couplings are needed only while factoring, before any solve
    C.flags = (int*)take(64);
    C.end = o;
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
        O.dsc[c] = !mixed ? 1.0 : in_f32_range(O.cd[c]) ? (double)rsqrtf((float)O.cd[c]) : 1.0 / sqrt(O.cd[c]);
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
// Waits for phase `parity` of the barrier for at most `limit` cycles (2^31,
// about a second, by default); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = 1LL << 31) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

}  // namespace
