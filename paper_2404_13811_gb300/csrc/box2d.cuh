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

// In-register Gauss-Jordan inverse of an SPD b x b block (row i in lane i),
// SPD so no pivoting.  The pivot row reaches every lane by shuffles from lane
// k; the pivot lane and the other lanes update with selects (no divergent
// paths), so a step is one chain of b shuffles and b FMAs.  Pivot
// reciprocals: the correctly rounded FP32 reciprocal in the FP32 form, FP64
// otherwise.  Writes Sout (row-major, b x b).
template <typename T, int BW>
__device__ void gj_invert(const T* S, T* Sout, int b, int* bad) {
    const int lane = threadIdx.x & 31;
    T a[BW];
#pragma unroll
    for (int c = 0; c < BW; ++c) a[c] = (lane < b && c < b) ? S[lane * b + c] : T(lane == c ? 1 : 0);
#pragma unroll
    for (int k = 0; k < BW; ++k) {
        if (k < b) {
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
            // one FMA per entry: the pivot lane computes 0 - (-ip) rv = ip rv,
            // the others a - f rv; column k takes ip / -f
            const bool isk = lane == k;
            const T f = a[k] * ip;
            const T fl = isk ? -ip : f;
#pragma unroll
            for (int c = 0; c < BW; ++c) {
                const T base = isk ? T(0) : a[c];
                a[c] = (c == k) ? (isk ? ip : -f) : base - fl * rv[c];
            }
        }
    }
    if (lane < b) {
#pragma unroll
        for (int c = 0; c < BW; ++c)
            if (c < b) Sout[lane * b + c] = a[c];
    }
    __syncwarp();
}

// Block LDL^T factorisation: Sinv[j] = S_j^{-1}.  cys / cxs: the scaled line
// / in-line couplings (type T, formed once).  The off-diagonal entries of
// each line Schur block are formed in T; its diagonal
// d_i - c_i^2 (S_{j-1}^{-1})_ii, where the cancellation is, in FP64 by one
// warp.  All threads participate; warp 0 inverts.
template <typename T, int BW>
__device__ void factor_box(const Box& B, const Ops& O, T* Sinv, T* cys, T* cxs, T* Sbuf, int* bad) {
    const int b = B.nx, nb = B.ny, bb = b * b;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int c = tid; c < B.n; c += nt) {
        cys[c] = (T)(O.cy[c] * O.dsc[c] * ((c + b < B.n) ? O.dsc[c + b] : 0.0));
        cxs[c] = (T)(-O.cx[c] * O.dsc[c] * ((c % b) < b - 1 ? O.dsc[c + 1] : 0.0));
    }
    __syncthreads();
    const int i0 = tid / b, k0 = tid - i0 * b;
    const int di = nt / b, dk = nt - di * b;
    for (int j = 0; j < nb; ++j) {
        const T* Sp = Sinv + (size_t)(j > 0 ? j - 1 : 0) * bb;
        int i = i0, k = k0;
        for (int t = tid; t < bb; t += nt) {
            if (i != k) {
                const int ci = j * b + i, ck = j * b + k;
                T s = T(0);
                if (k == i + 1) s = cxs[ci];
                else if (k == i - 1) s = cxs[ck];
                if (j > 0) s -= cys[ci - b] * Sp[i * b + k] * cys[ck - b];
                Sbuf[t] = s;
            }
            k += dk;
            i += di;
            if (k >= b) {
                k -= b;
                ++i;
            }
        }
        if (tid < b) {
            const int ci = j * b + tid;
            double s = O.cd[ci] * O.dsc[ci] * O.dsc[ci];
            if (j > 0) {
                const double cc = (double)cys[ci - b];
                s -= cc * cc * (double)Sp[tid * b + tid];
            }
            Sbuf[tid * b + tid] = (T)s;
        }
        __syncthreads();
        if (tid < 32) gj_invert<T, BW>(Sbuf, Sinv + (size_t)j * bb, b, bad);
        __syncthreads();
    }
}

// One warp sweeps in place: on entry w holds the scaled right-hand side, on
// exit the scaled solution.  The FP32 form reads rows of the symmetric line
// blocks as float4 (warp_sweeps_f32, after the CTA-wide helpers below).
__device__ void warp_sweeps_f32(const float* __restrict__ Sinv, const float* __restrict__ cys, float* w, float* z,
                                int b, int nb);

template <typename T>
__device__ void warp_sweeps(const T* __restrict__ Sinv, const T* __restrict__ cys, T* w, T* zbuf,
                            int b, int nb) {
    if constexpr (std::is_same<T, float>::value) {
        if ((b & 3) == 0) {
            warp_sweeps_f32(Sinv, cys, w, zbuf, b, nb);
            return;
        }
    }
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

// The same two sweeps with the whole CTA on one right-hand side: warp q
// reduces columns [q kq, (q + 1) kq) of each line block; the partial sums of
// the warps meet in red (double-buffered by line parity, so one barrier per
// line), and every warp forms the next line's input in its own zw (32
// entries per warp).  w: scaled right-hand side in, scaled solution out.
// FP32 sweeps of a CTA-wide solve, by warp 0 alone (no block barrier per
// line; one warp is limited by the latency of the line-to-line exchange,
// a 4-warp split by its barrier): lane i owns row i of the line (b <= 32).
// The local operator is symmetric, so every block of S^-1 is too, and lane
// i reads row i of the block -- with b a multiple of 4, as b / 4 float4
// loads issued before the line's input is ready; otherwise column i by
// scalar loads.  The line input goes through z (32 entries, zero beyond b)
// and comes back as float4 broadcasts; four accumulators.  The other warps
// wait at the closing barrier.
__device__ __forceinline__ float sline_row_dot(const float* __restrict__ S, const float* z, int b, int lane,
                                               float4 (&s4)[8]) {
    float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (4 * q < b) {
            const float4 zz = reinterpret_cast<const float4*>(z)[q];
            a[0] += s4[q].x * zz.x;
            a[1] += s4[q].y * zz.y;
            a[2] += s4[q].z * zz.z;
            a[3] += s4[q].w * zz.w;
        }
    return (a[0] + a[1]) + (a[2] + a[3]);
}

__device__ __forceinline__ void load_srow(float4 (&s4)[8], const float* __restrict__ S, int b, int lane) {
    const float4* Sr = reinterpret_cast<const float4*>(S + (lane < b ? lane : 0) * b);
#pragma unroll
    for (int q = 0; q < 8; ++q) s4[q] = 4 * q < b ? Sr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float sline_col_dot(const float* __restrict__ S, const float* z, int b, int lane) {
    float a0 = 0.f, a1 = 0.f;
    if (lane < b) {
        int k = 0;
        for (; k + 1 < b; k += 2) {
            a0 += S[k * b + lane] * z[k];
            a1 += S[(k + 1) * b + lane] * z[k + 1];
        }
        if (k < b) a0 += S[k * b + lane] * z[k];
    }
    return a0 + a1;
}

__device__ void warp0_sweeps(const float* __restrict__ Sinv, const float* __restrict__ cys, float* w, float* z,
                             int b, int nb) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const size_t bb = (size_t)b * b;
        const bool rows = (b & 3) == 0;
        float4 s4[8];
        float cur = 0.f;
        // forward: w_j <- S_j^-1 (w_j + cys_{j-1} w_{j-1})
        for (int j = 0; j < nb; ++j) {
            if (rows) load_srow(s4, Sinv + j * bb, b, lane);
            float zj = 0.f;
            if (lane < b) zj = w[j * b + lane] + (j > 0 ? cys[(j - 1) * b + lane] * cur : 0.f);
            z[lane] = zj;
            __syncwarp();
            cur = rows ? sline_row_dot(Sinv + j * bb, z, b, lane, s4) : sline_col_dot(Sinv + j * bb, z, b, lane);
            if (lane < b) w[j * b + lane] = cur;
            __syncwarp();
        }
        // backward: w_j <- w_j + S_j^-1 cys_j w_{j+1}
        for (int j = nb - 2; j >= 0; --j) {
            if (rows) load_srow(s4, Sinv + j * bb, b, lane);
            z[lane] = lane < b ? cys[j * b + lane] * cur : 0.f;
            const float wf = lane < b ? w[j * b + lane] : 0.f;
            __syncwarp();
            cur = wf + (rows ? sline_row_dot(Sinv + j * bb, z, b, lane, s4) : sline_col_dot(Sinv + j * bb, z, b, lane));
            if (lane < b) w[j * b + lane] = cur;
            __syncwarp();
        }
    }
    __syncthreads();
}

// The FP32 sweeps of one warp (as warp0_sweeps, b a multiple of 4) for a
// warp that owns its right-hand side; no block barrier.
__device__ void warp_sweeps_f32(const float* __restrict__ Sinv, const float* __restrict__ cys, float* w, float* z,
                                int b, int nb) {
    const int lane = threadIdx.x & 31;
    const size_t bb = (size_t)b * b;
    float4 s4[8];
    float cur = 0.f;
    for (int j = 0; j < nb; ++j) {
        load_srow(s4, Sinv + j * bb, b, lane);
        float zj = 0.f;
        if (lane < b) zj = w[j * b + lane] + (j > 0 ? cys[(j - 1) * b + lane] * cur : 0.f);
        z[lane] = zj;
        __syncwarp();
        cur = sline_row_dot(Sinv + j * bb, z, b, lane, s4);
        if (lane < b) w[j * b + lane] = cur;
        __syncwarp();
    }
    for (int j = nb - 2; j >= 0; --j) {
        load_srow(s4, Sinv + j * bb, b, lane);
        z[lane] = lane < b ? cys[j * b + lane] * cur : 0.f;
        const float wf = lane < b ? w[j * b + lane] : 0.f;
        __syncwarp();
        cur = wf + sline_row_dot(Sinv + j * bb, z, b, lane, s4);
        if (lane < b) w[j * b + lane] = cur;
        __syncwarp();
    }
}

template <typename T>
__device__ void cta_sweeps(const T* __restrict__ Sinv, const T* __restrict__ cys, T* w, T* zw, T* red, int b,
                           int nb) {
    if constexpr (std::is_same<T, float>::value) {
        warp0_sweeps(Sinv, cys, w, zw, b, nb);
        return;
    }
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5, nq = blockDim.x >> 5;
    const int kq = (b + nq - 1) / nq, ka = wq * kq, kb = min(b, ka + kq);
    T* z = zw + wq * 32;
    int par = 0;
    T cur = T(0);   // this lane's entry of the last finished line
    // forward: w_j <- S_j^-1 (w_j + cys_{j-1} w_{j-1})
    for (int j = 0; j < nb; ++j) {
        if (lane < b) z[lane] = w[j * b + lane] + (j > 0 ? cys[(j - 1) * b + lane] * cur : T(0));
        __syncwarp();
        T acc = T(0);
        if (lane < b) {
            const T* S = Sinv + (size_t)j * b * b;
            for (int k = ka; k < kb; ++k) acc += S[k * b + lane] * z[k];
            red[(par * nq + wq) * 32 + lane] = acc;
        }
        __syncthreads();
        if (lane < b) {
            T s = T(0);
            for (int q = 0; q < nq; ++q) s += red[(par * nq + q) * 32 + lane];
            cur = s;
            if (wq == 0) w[j * b + lane] = s;
        }
        par ^= 1;
        __syncwarp();
    }
    // backward: w_j <- w_j + S_j^-1 cys_j w_{j+1}
    for (int j = nb - 2; j >= 0; --j) {
        if (lane < b) z[lane] = cys[j * b + lane] * cur;
        // this line's forward value, read by every warp before warp 0 overwrites it
        const T wf = lane < b ? w[j * b + lane] : T(0);
        __syncwarp();
        T acc = T(0);
        if (lane < b) {
            const T* S = Sinv + (size_t)j * b * b;
            for (int k = ka; k < kb; ++k) acc += S[k * b + lane] * z[k];
            red[(par * nq + wq) * 32 + lane] = acc;
        }
        __syncthreads();
        if (lane < b) {
            T s = wf;
            for (int q = 0; q < nq; ++q) s += red[(par * nq + q) * 32 + lane];
            cur = s;
            if (wq == 0) w[j * b + lane] = s;
        }
        par ^= 1;
        __syncwarp();
    }
    __syncthreads();
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
    size_t o = align16(tsz * n * nx);
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
    T* Sbuf;
    T* zbuf;   // NWARP * 32
    double* bsrc; // n: fixed right-hand side of the particular problem
    double* X; // nrhs * n
    T* W;      // nrhs * n
    int* flags;
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
    s += align16(sizeof(T) * n * nx) + align16(sizeof(T) * n) * 2 + align16(sizeof(T) * nx * nx);
    s += align16(sizeof(T) * 32 * NWARP) + (part ? align16(sizeof(double) * n) : 0);
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
    C.Sinv = (T*)take(sizeof(T) * n * nx);
    C.cys = (T*)take(sizeof(T) * n);
    C.cxs = (T*)take(sizeof(T) * n);
    C.Sbuf = (T*)take(sizeof(T) * nx * nx);
    C.zbuf = (T*)take(sizeof(T) * 32 * NWARP);
    C.bsrc = part ? (double*)take(sizeof(double) * n) : nullptr;
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
