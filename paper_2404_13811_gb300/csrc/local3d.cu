// 3D local Robin/Darcy solves of MRCM-OS on sm_103a.
//
// One CTA (256 threads) per job (a subdomain box).  The cell-centred RT0
// operator of the box (Sec. 2.2; the face laws of Eq. (genRobin)) is block
// tridiagonal over the planes normal to the box's longest axis a2; a plane
// has b = n_a0 n_a1 cells (a0 fastest) and planes couple through diagonal
// blocks D_j (the a2-face transmissibilities).  The factorisation
// (Algorithm 1, Steps 1 and 6) keeps the inverses of the plane Schur
// complements S_j = A_jj - D_{j-1} S_{j-1}^{-1} D_{j-1}: each S_j is formed
// in shared memory from S_{j-1}^{-1} in place (D is diagonal) and inverted
// there by the whole CTA (Gauss-Jordan, SPD so no pivoting); the inverses go
// to global memory (a box's factor, n_a2 b^2 entries, does not fit on chip).
// A solve is two sweeps of dense b x b products, all right-hand sides of a
// round at once, so each plane inverse is read once per sweep.
//
// Precision: T = double is the FP64 form.  T = float is the mixed form:
// Jacobi-scaled operator, Schur diagonals and pivot reciprocals from FP64,
// FP32 sweeps, FP64 residual refinement to ir_tol (as in 2D).
#include "box2d.cuh"

namespace {

constexpr int T3 = 256;   // threads per CTA
constexpr int NR3 = 4;    // right-hand sides per round
constexpr int CR3 = 16;   // rows of a plane inverse per streamed chunk

// plane stride of a kept factor: b^2 entries padded to 16 bytes
__host__ __device__ __forceinline__ size_t plane_stride(int b) { return ((size_t)b * b + 3) & ~size_t(3); }
// entries of one staging buffer for `rows` rows of a plane: a multiple of 4
// entries, so that the second buffer starts on a 16-byte boundary (the bulk
// copy needs 16-byte aligned destinations) and the copy size, rounded up to
// 16 bytes, fits
__host__ __device__ __forceinline__ size_t stage_cap(int rows, int b) {
    return (((size_t)rows * b + 3) & ~size_t(3)) + 4;
}

struct Box3 {
    int lo[3], hi[3], n[3];
    int nc;
    int a0, a1, a2;   // in-plane axes (a0 fastest) and the plane axis
    int b, np;        // plane size, number of planes
    int kind[6];      // 0 Neumann, 1 Dirichlet, 2 Robin
    double val[6];
    double alpha;
    int ts[6], tt[6]; // tangential axes (ascending) of each side
    int soff[7];      // offsets of the sides in the boundary-face arrays
    int crows;        // rows of a plane inverse per streamed copy
};

// rows per streamed copy: whole planes in the mixed form (two plane buffers
// keep ~64 KB in flight per SM), 16-row chunks in the FP64 form
__host__ __device__ __forceinline__ int stream_rows(int b, bool mixed) { return mixed ? b : (b < CR3 ? b : CR3); }

__device__ void setup_box3(Box3& B, const MemberDev& md, const int* lo, const int* hi, double alpha) {
    for (int a = 0; a < 3; ++a) {
        B.lo[a] = lo[a];
        B.hi[a] = hi[a];
        B.n[a] = hi[a] - lo[a];
    }
    B.nc = B.n[0] * B.n[1] * B.n[2];
    int a2 = 2;
    for (int a = 1; a >= 0; --a)
        if (B.n[a] > B.n[a2]) a2 = a;
    B.a2 = a2;
    B.a0 = a2 == 0 ? 1 : 0;
    B.a1 = a2 == 2 ? 1 : 2;
    B.b = B.n[B.a0] * B.n[B.a1];
    B.np = B.n[a2];
    B.alpha = alpha;
    B.soff[0] = 0;
    for (int sid = 0; sid < 6; ++sid) {
        const int a = sid >> 1;
        const bool phys = (sid & 1) ? (hi[a] == md.n[a]) : (lo[a] == 0);
        if (phys) {
            B.kind[sid] = md.bc_kind[sid] == 1 ? 1 : 0;
            B.val[sid] = md.bc_val[sid];
        } else {
            B.kind[sid] = 2;
            B.val[sid] = 0.0;
        }
        B.ts[sid] = a == 0 ? 1 : 0;
        B.tt[sid] = a == 2 ? 1 : 2;
        B.soff[sid + 1] = B.soff[sid] + B.n[B.ts[sid]] * B.n[B.tt[sid]];
    }
}

// natural coordinates of the cell at block index t
__device__ __forceinline__ void bcoord(const Box3& B, int t, int* c) {
    const int j = t / B.b, pos = t - j * B.b;
    c[B.a2] = j;
    c[B.a1] = pos / B.n[B.a0];
    c[B.a0] = pos - c[B.a1] * B.n[B.a0];
}
__device__ __forceinline__ int bidx(const Box3& B, const int* c) {
    return c[B.a2] * B.b + c[B.a0] + B.n[B.a0] * c[B.a1];
}
__device__ __forceinline__ long long gidx(const Box3& B, const MemberDev& md, const int* c) {
    return (B.lo[0] + c[0]) + (long long)md.n[0] * ((B.lo[1] + c[1]) + (long long)md.n[1] * (B.lo[2] + c[2]));
}
__device__ __forceinline__ long long gstride(const MemberDev& md, int a) {
    return a == 0 ? 1LL : a == 1 ? (long long)md.n[0] : (long long)md.n[0] * md.n[1];
}
// face index of a cell on side sid (first tangential axis fastest)
__device__ __forceinline__ int side_e(const Box3& B, int sid, const int* c) {
    return c[B.ts[sid]] + B.n[B.ts[sid]] * c[B.tt[sid]];
}
// P0 / P1 function m on a side face with tangential coordinates (cs, ct)
// relative to a side of extents (ls, lt): 1, s, t in [-1, 1]
__device__ __forceinline__ double psi3(int m, int cs, int ls, int ct, int lt) {
    return m == 0 ? 1.0 : m == 1 ? (double)(2 * cs + 1 - ls) / ls : (double)(2 * ct + 1 - lt) / lt;
}

struct Ops3 {
    double *cd, *c0, *c1, *c2, *dsc;  // diagonal, couplings to +a0, +a1, +a2, Jacobi scale (block order)
    double *bT, *bB;                   // boundary-face transmissibility and Robin beta per side face
    unsigned char* nb;                 // neighbour bits: 1 -a0, 2 +a0, 4 -a1, 8 +a1, 16 -a2, 32 +a2
};

__device__ void build_ops3(const Box3& B, const MemberDev& md, const DevPtrs& P, Ops3& O, bool mixed) {
    const double* Tf = P.Tf + md.cell_off * 3;
    const double* hkg = P.hk + md.cell_off * 3;
    const double* wh = P.wh + md.cell_off * 3;
    const double vol = md.h[0] * md.h[1] * md.h[2];
    for (int t = threadIdx.x; t < B.nc; t += blockDim.x) {
        int c[3];
        bcoord(B, t, c);
        const long long g = gidx(B, md, c);
        O.c0[t] = c[B.a0] < B.n[B.a0] - 1 ? Tf[g * 3 + B.a0] : 0.0;
        O.c1[t] = c[B.a1] < B.n[B.a1] - 1 ? Tf[g * 3 + B.a1] : 0.0;
        O.c2[t] = c[B.a2] < B.n[B.a2] - 1 ? Tf[g * 3 + B.a2] : 0.0;
        unsigned char m = 0;
        if (c[B.a0] > 0) m |= 1;
        if (c[B.a0] < B.n[B.a0] - 1) m |= 2;
        if (c[B.a1] > 0) m |= 4;
        if (c[B.a1] < B.n[B.a1] - 1) m |= 8;
        if (c[B.a2] > 0) m |= 16;
        if (c[B.a2] < B.n[B.a2] - 1) m |= 32;
        O.nb[t] = m;
    }
    for (int sid = 0; sid < 6; ++sid) {
        const int a = sid >> 1;
        const int ls = B.n[B.ts[sid]];
        const int faces = B.soff[sid + 1] - B.soff[sid];
        const double area = vol / md.h[a];
        for (int e = threadIdx.x; e < faces; e += blockDim.x) {
            int c[3];
            c[a] = (sid & 1) ? B.n[a] - 1 : 0;
            c[B.ts[sid]] = e % ls;
            c[B.tt[sid]] = e / ls;
            const long long g = gidx(B, md, c);
            const double hin = hkg[g * 3 + a];
            double T = 0.0, beta = 0.0;
            if (B.kind[sid] == 2) {
                const long long gf = (sid & 1) ? g : g - gstride(md, a);
                beta = B.alpha * wh[gf * 3 + a];
                T = area * rcp64(hin + beta);
            } else if (B.kind[sid] == 1) {
                T = area * rcp64(hin);
            }
            O.bT[B.soff[sid] + e] = T;
            O.bB[B.soff[sid] + e] = beta;
        }
    }
    __syncthreads();
    const int s0 = 1, s1 = B.n[B.a0], s2 = B.b;
    for (int t = threadIdx.x; t < B.nc; t += blockDim.x) {
        const unsigned char m = O.nb[t];
        double d = O.c0[t] + O.c1[t] + O.c2[t];
        if (m & 1) d += O.c0[t - s0];
        if (m & 4) d += O.c1[t - s1];
        if (m & 16) d += O.c2[t - s2];
        if ((m & 63) != 63) {
            int c[3];
            bcoord(B, t, c);
            for (int sid = 0; sid < 6; ++sid) {
                const int a = sid >> 1;
                if (c[a] == ((sid & 1) ? B.n[a] - 1 : 0)) d += O.bT[B.soff[sid] + side_e(B, sid, c)];
            }
        }
        O.cd[t] = d;
        if (mixed) O.dsc[t] = in_f32_range(d) ? (double)rsqrtf((float)d) : 1.0 / sqrt(d);
    }
    __syncthreads();
}

// (A x)_t of the unscaled FP64 operator with the couplings read from the
// global face coefficients (the mixed form keeps no coupling arrays on chip
// during the solves)
__device__ __forceinline__ double applyA3g(const Box3& B, const MemberDev& md, const double* __restrict__ Tf,
                                           const double* cd, const unsigned char* nbits, const double* x, int t) {
    int c[3];
    bcoord(B, t, c);
    const long long g = gidx(B, md, c);
    const unsigned char m = nbits[t];
    const int s1 = B.n[B.a0], s2 = B.b;
    double s = cd[t] * x[t];
    if (m & 1) s -= Tf[(g - gstride(md, B.a0)) * 3 + B.a0] * x[t - 1];
    if (m & 2) s -= Tf[g * 3 + B.a0] * x[t + 1];
    if (m & 4) s -= Tf[(g - gstride(md, B.a1)) * 3 + B.a1] * x[t - s1];
    if (m & 8) s -= Tf[g * 3 + B.a1] * x[t + s1];
    if (m & 16) s -= Tf[(g - gstride(md, B.a2)) * 3 + B.a2] * x[t - s2];
    if (m & 32) s -= Tf[g * 3 + B.a2] * x[t + s2];
    return s;
}

// 16-byte vectors of the shared-memory kernels (float4 / double2)
template <typename T> struct V16;
template <> struct V16<float> {
    using V = float4;
    static constexpr int W = 4;
};
template <> struct V16<double> {
    using V = double2;
    static constexpr int W = 2;
};
template <typename T>
union VU {
    typename V16<T>::V v;
    T a[V16<T>::W];
};

// leading dimension of the shared plane block: b padded to 4 entries
__host__ __device__ __forceinline__ int plane_ld(int b) { return (b + 3) & ~3; }

// In-place Gauss-Jordan inverse of an SPD b x b matrix in shared memory by
// the whole CTA (row-major, leading dimension ld = plane_ld(b), padding
// columns zero).  Each thread updates 16-byte groups of a row.  Pivot
// reciprocals from the FP64 pivot.
template <typename T>
__device__ void gj_cta(T* S, int b, int ld, T* rowbuf, T* colbuf, T* ipb, int* bad) {
    constexpr int W = V16<T>::W;
    using V = typename V16<T>::V;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ng = ld / W;                 // groups per row
    const int tot = b * ng;
    const int i0 = tid / ng, g0 = tid - i0 * ng;
    const int di = nt / ng, dg = nt - di * ng;
    for (int k = 0; k < b; ++k) {
        if (tid == 0) {
            double piv = (double)S[k * ld + k];
            if (!(piv > 0.0)) {
                *bad = 1;
                piv = 1.0;
            }
            *ipb = std::is_same<T, float>::value ? (T)__frcp_rn((float)piv) : (T)rcp64(piv);
        }
        for (int t = tid; t < ld; t += nt) {
            rowbuf[t] = S[k * ld + t];
            if (t < b) colbuf[t] = S[t * ld + k];
        }
        __syncthreads();
        const T ip = *ipb;
        const int gk = k / W, ek = k - gk * W;
        int i = i0, g = g0;
        for (int t = tid; t < tot; t += nt) {
            VU<T> x, r;
            x.v = *reinterpret_cast<const V*>(&S[i * ld + g * W]);
            r.v = *reinterpret_cast<const V*>(&rowbuf[g * W]);
            const bool colk = g == gk;
            if (i == k) {
#pragma unroll
                for (int e = 0; e < W; ++e) x.a[e] = (colk && e == ek) ? ip : r.a[e] * ip;
            } else {
                const T f = colbuf[i] * ip;
#pragma unroll
                for (int e = 0; e < W; ++e) x.a[e] = (colk && e == ek) ? -f : x.a[e] - f * r.a[e];
            }
            *reinterpret_cast<V*>(&S[i * ld + g * W]) = x.v;
            g += dg;
            i += di;
            if (g >= ng) {
                g -= ng;
                ++i;
            }
        }
        __syncthreads();
    }
}

// Block LDL^T over planes; inverses of the plane Schur complements to F
// (row stride b, plane stride plane_stride(b)).  Sb: ld = plane_ld(b).
template <typename T>
__device__ void factor3(const Box3& B, const Ops3& O, const T* c2s, T* F, T* Sb, T* rowbuf, T* colbuf, T* ipb,
                        int* bad, bool mixed) {
    const int b = B.b, ld = plane_ld(b), bb = b * b;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int i0 = tid / b, k0 = tid - i0 * b;
    const int di = nt / b, dk = nt - di * b;
    const int n0 = B.n[B.a0];
    for (int t = tid; t < b * ld; t += nt) Sb[t] = T(0);   // padding columns stay zero
    __syncthreads();
    for (int j = 0; j < B.np; ++j) {
        int i = i0, k = k0;
        for (int t = tid; t < bb; t += nt) {
            const int ci = j * b + i, ck = j * b + k;
            const int sidx = i * ld + k;
            const double si = mixed ? O.dsc[ci] : 1.0;
            if (i == k) {
                double s = O.cd[ci] * si * si;
                if (j > 0) {
                    const double cc = (double)c2s[ci - b];
                    s -= cc * (cc * (double)Sb[sidx]);   // not cc^2 (range at tiny couplings)
                }
                Sb[sidx] = (T)s;
            } else {
                const double sk = mixed ? O.dsc[ck] : 1.0;
                T s = T(0);
                if (k == i + 1 && (O.nb[ci] & 2)) s = (T)(-O.c0[ci] * si * sk);
                else if (k == i - 1 && (O.nb[ci] & 1)) s = (T)(-O.c0[ck] * si * sk);
                else if (k == i + n0) s = (T)(-O.c1[ci] * si * sk);
                else if (k == i - n0) s = (T)(-O.c1[ck] * si * sk);
                if (j > 0) s -= c2s[ci - b] * Sb[sidx] * c2s[ck - b];
                Sb[sidx] = s;
            }
            k += dk;
            i += di;
            if (k >= b) {
                k -= b;
                ++i;
            }
        }
        __syncthreads();
        gj_cta<T>(Sb, b, ld, rowbuf, colbuf, ipb, bad);
        T* Fj = F + (size_t)j * plane_stride(b);
        {
            int ii = i0, kk = k0;
            for (int t = tid; t < bb; t += nt) {
                Fj[t] = Sb[ii * ld + kk];
                kk += dk;
                ii += di;
                if (kk >= b) {
                    kk -= b;
                    ++ii;
                }
            }
        }
        // the solves read the factor through the bulk-copy (async) proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();
    }
}

// Two sweeps over the planes for nr right-hand sides in W ([nr][nc], block
// order): on entry the scaled right-hand sides, on exit the scaled
// solutions.  The plane inverses (symmetric, row-major, plane stride padded
// to 16 bytes) stream from global memory through the bulk-copy (TMA) engine
// in chunks of B.crows rows into two shared buffers: chunk s + 1 is in flight
// while chunk s is used.  The sweep input of a plane is kept interleaved
// (vb[c][4], all right-hand sides of a column in one 16-byte load).  For
// b <= T3/2 the two halves of the CTA take the two halves of each chunk and
// meet in red (which reuses vb once a plane is done); otherwise one thread
// per row.  Returns false when a copy did
// not complete in time (the CTA then stops using the buffers).
template <typename T>
__device__ bool sweeps3(const Box3& B, const T* __restrict__ F, const T* __restrict__ c2s, T* W, T* vb, T* cbuf,
                        T* red, uint64_t* bar, uint32_t* par, int nr) {
    const int b = B.b, nc = B.nc;
    const int tid = threadIdx.x, nt = blockDim.x;
    const size_t ps = plane_stride(b);
    const int CRr = B.crows;
    const int nch = (b + CRr - 1) / CRr;
    const int nplane = 2 * B.np - 1;                  // forward planes, then backward planes np-2 .. 0
    const int total = nplane * nch;
    const size_t cap = stage_cap(CRr, b);              // entries per buffer
    const bool split = b <= nt / 2;
    const int r = split ? tid % (nt / 2) : tid;        // row of this thread (active if r < b)
    const int hf = split ? tid / (nt / 2) : 0;         // half of each chunk
    auto plane_of = [&](int p) { return p < B.np ? p : 2 * B.np - 2 - p; };
    auto issue = [&](int st) {
        const int j = plane_of(st / nch), ci = st % nch;
        const int c0 = ci * CRr, cr = min(CRr, b - c0);
        const uint32_t bytes = (uint32_t)((sizeof(T) * (size_t)cr * b + 15) & ~size_t(15));
        T* dst = cbuf + (size_t)(st & 1) * cap;
        mbar_expect_tx(&bar[st & 1], bytes);
        bulk_g2s(dst, F + (size_t)j * ps + (size_t)c0 * b, bytes, &bar[st & 1]);
    };
    if (tid == 0) issue(0);
    T acc[NR3];
    bool ok = true;
    for (int st = 0; st < total; ++st) {
        const int p = st / nch, ci = st % nch, j = plane_of(p);
        const bool fwd = p < B.np;
        if (ci == 0) {
            for (int c = tid; c < b; c += nt) {
#pragma unroll
                for (int q = 0; q < NR3; ++q) {
                    T v = T(0);
                    if (q < nr) {
                        if (fwd) {
                            v = W[q * nc + j * b + c];
                            if (j > 0) v += c2s[(j - 1) * b + c] * W[q * nc + (j - 1) * b + c];
                        } else {
                            v = c2s[j * b + c] * W[q * nc + (j + 1) * b + c];
                        }
                    }
                    vb[c * NR3 + q] = v;
                }
            }
#pragma unroll
            for (int q = 0; q < NR3; ++q) acc[q] = T(0);
        }
        const bool done = mbar_wait(&bar[st & 1], par[st & 1]);
        par[st & 1] ^= 1u;
        if (__syncthreads_or(!done)) {
            // the copy of step st is late: wait once more (bounded) so that no
            // copy targets the buffer after the CTA stops using it
            ok = false;
            if (tid == 0) mbar_wait(&bar[st & 1], par[st & 1] ^ 1u);
            break;
        }
        if (tid == 0 && st + 1 < total) issue(st + 1);
        const T* S = cbuf + (size_t)(st & 1) * cap;
        const int c0 = ci * CRr, cr = min(CRr, b - c0);
        if (r < b) {
            int ca = 0, cb = cr;
            if (split) {
                const int hc = (cr + 1) / 2;
                ca = hf * hc;
                cb = min(cr, ca + hc);
            }
            for (int c = ca; c < cb; ++c) {
                const T sv = S[c * b + r];
                const T* vq = vb + (size_t)(c0 + c) * NR3;
                if (NR3 == 4 && std::is_same<T, float>::value) {
                    const float4 v4 = *reinterpret_cast<const float4*>(vq);
                    acc[0] += sv * (T)v4.x;
                    acc[1] += sv * (T)v4.y;
                    acc[2] += sv * (T)v4.z;
                    acc[3] += sv * (T)v4.w;
                } else {
#pragma unroll
                    for (int q = 0; q < NR3; ++q) acc[q] += sv * vq[q];
                }
            }
        }
        if (ci == nch - 1) {
            if (split) {
                __syncthreads();   // red shares memory with vb: every thread is done reading vb
                if (hf == 1 && r < b)
#pragma unroll
                    for (int q = 0; q < NR3; ++q) red[r * NR3 + q] = acc[q];
                __syncthreads();
            }
            if (hf == 0 && r < b) {
#pragma unroll
                for (int q = 0; q < NR3; ++q) {
                    if (q >= nr) continue;
                    const T v = split ? acc[q] + red[r * NR3 + q] : acc[q];
                    if (fwd) W[q * nc + j * b + r] = v;
                    else W[q * nc + j * b + r] += v;
                }
            }
        }
        __syncthreads();
    }
    return ok;
}

__device__ __forceinline__ void atomic_max_f(unsigned int* a, float v) { atomicMax(a, __float_as_uint(v)); }

// Solves A x_q = rhs_q for nr right-hand sides with the whole CTA: sweeps
// with the kept factor (FP32 in the mixed form, FP64 in the FP64 form) and
// refinement with FP64 residuals of the unscaled operator, the iterate X in
// FP64.  High-contrast boxes reach a residual floor above what a fixed
// tolerance can ask for, so the refinement runs to that floor: it stops when
// every right-hand side has |r| <= 1e-3 ir_tol |b| (scaled max norms), or has
// |r| <= ir_tol |b| and no longer halves its residual per step.  The FP64 form
// (a direct solve, then refinement with the same rule, at most 4 sweep
// pairs) never reports non-convergence.  Returns the number of sweep pairs.
template <typename T, typename Rhs>
__device__ int solve3(const Box3& B, const MemberDev& md, const double* Tfm, const Ops3& O, const T* F, const T* c2s,
                      double* X, T* W, T* vb, T* cbuf, T* red, uint64_t* bar, uint32_t* par, unsigned int* nrm, int nr,
                      const Rhs& rhs, double tol, int max_ir, int* noconv, int* bad) {
    constexpr bool mixed = std::is_same<T, float>::value;
    const int nc = B.nc, tid = threadIdx.x, nt = blockDim.x;
    if (*bad) return 0;   // a staged copy failed earlier: the buffers are not usable
    const int mit = mixed ? max_ir : 4;
    if (tid < 3 * NR3) nrm[tid] = tid < NR3 ? 0u : 0x7f800000u;   // |b|, then |r| of the previous step (inf)
    __syncthreads();
    for (int q = 0; q < nr; ++q)
        for (int t = tid; t < nc; t += nt) {
            const double v = (mixed ? O.dsc[t] : 1.0) * rhs(q, t);
            X[q * nc + t] = 0.0;
            W[q * nc + t] = (T)v;
            atomic_max_f(&nrm[q], fabsf((float)v));
        }
    __syncthreads();
    int it = 0;
    for (; it < mit; ++it) {
        if (!sweeps3<T>(B, F, c2s, W, vb, cbuf, red, bar, par, nr)) {
            if (threadIdx.x == 0) *bad = 1;
            __syncthreads();
            break;
        }
        for (int q = 0; q < nr; ++q)
            for (int t = tid; t < nc; t += nt) X[q * nc + t] += (mixed ? O.dsc[t] : 1.0) * (double)W[q * nc + t];
        if (tid < NR3) nrm[NR3 + tid] = 0u;
        __syncthreads();
        for (int q = 0; q < nr; ++q)
            for (int t = tid; t < nc; t += nt) {
                const double v = (mixed ? O.dsc[t] : 1.0) * (rhs(q, t) - applyA3g(B, md, Tfm, O.cd, O.nb, X + q * nc, t));
                W[q * nc + t] = (T)v;
                atomic_max_f(&nrm[NR3 + q], fabsf((float)v));
            }
        __syncthreads();
        bool done = true, reached = true;
        for (int q = 0; q < nr; ++q) {
            const double bn = (double)__uint_as_float(nrm[q]), rn = (double)__uint_as_float(nrm[NR3 + q]);
            const double rp = (double)__uint_as_float(nrm[2 * NR3 + q]);
            const bool ok = bn == 0.0 || rn <= 1e-3 * tol * bn || (rn <= tol * bn && rn > 0.5 * rp);
            if (!ok) done = false;
            if (!(bn == 0.0 || rn <= tol * bn)) reached = false;
        }
        __syncthreads();
        if (tid < NR3) nrm[2 * NR3 + tid] = nrm[NR3 + tid];
        if (done) {
            ++it;
            break;
        }
        if (it == mit - 1 && !reached && tid == 0 && mixed) *noconv = 1;
    }
    __syncthreads();
    return it;
}

// f |c| + Dirichlet / Neumann data + Robin data lam (may be null) of cell t
__device__ double source_rhs3(const Box3& B, const Ops3& O, const MemberDev& md, const double* fm, const double* lam,
                              int t) {
    int c[3];
    bcoord(B, t, c);
    const double vol = md.h[0] * md.h[1] * md.h[2];
    double r = fm[gidx(B, md, c) - 0] * vol;
    if ((O.nb[t] & 63) != 63) {
        for (int sid = 0; sid < 6; ++sid) {
            const int a = sid >> 1;
            if (c[a] != ((sid & 1) ? B.n[a] - 1 : 0)) continue;
            const int e = B.soff[sid] + side_e(B, sid, c);
            if (B.kind[sid] == 1) r += O.bT[e] * B.val[sid];
            else if (B.kind[sid] == 0) r -= vol / md.h[a] * B.val[sid];
            else if (lam) r += O.bT[e] * lam[e];
        }
    }
    return r;
}

// Right-hand sides of a group of basis solves; sk[q] < 0 marks the particular
// problem on hat-Omega_i (a variant of Step 4), whose vector bs is stored.
struct RhsBasis3 {
    const Box3* B;
    const double* bT;
    const double* bs;
    int sk[NR3], mk[NR3];
    __device__ double operator()(int q, int t) const {
        if (sk[q] < 0) return bs[t];
        const int sid = sk[q], a = sid >> 1;
        int c[3];
        bcoord(*B, t, c);
        if (c[a] != ((sid & 1) ? B->n[a] - 1 : 0)) return 0.0;
        const int ts = B->ts[sid], tt = B->tt[sid];
        return bT[B->soff[sid] + side_e(*B, sid, c)] * psi3(mk[q], c[ts], B->n[ts], c[tt], B->n[tt]);
    }
};

struct RhsStored3 {
    const double* b;
    __device__ double operator()(int, int t) const { return b[t]; }
};

// Shared-memory layout.  Persistent: diagonal, neighbour bits, scaled plane
// coupling, boundary faces, Robin data, stored right-hand side and (mixed
// form) the FP32 work vectors W and the sweep input vb.  Overlaid: the
// factor phase (the plane Schur block and, in the mixed form, the in-plane
// couplings) and the solve phase (the streamed plane buffers; in the FP64
// form also W and vb).  The FP64 iterates live in global scratch (one slot
// per CTA).  The mixed form streams whole planes, the FP64 form 16-row
// chunks.
__host__ __device__ inline void box3_dims(int nx, int ny, int nz, int* b, int* npl) {
    int n[3] = {nx, ny, nz};
    int a2 = 2;
    for (int a = 1; a >= 0; --a)
        if (n[a] > n[a2]) a2 = a;
    *b = nx * ny * nz / n[a2];
    *npl = n[a2];
}

__host__ __device__ inline size_t carve3_bytes(int tsz, int nx, int ny, int nz, bool stored_rhs) {
    int b, npl;
    box3_dims(nx, ny, nz, &b, &npl);
    const bool mixed = tsz == 4;
    const size_t nc = (size_t)nx * ny * nz;
    const size_t per = 2 * ((size_t)nx * ny + (size_t)ny * nz + (size_t)nx * nz);
    const size_t crw = (size_t)stream_rows(b, mixed);
    size_t s = align16(sizeof(double) * nc);                                  // cd
    if (mixed) s += align16(sizeof(double) * nc) + align16(tsz * nc);         // dsc c2s
    else s += align16(sizeof(double) * nc) * 3;                               // c0 c1 c2
    s += align16(nc);                                                          // nb
    s += align16(sizeof(double) * per) * 3;                                    // bT bB lam
    s += stored_rhs ? align16(sizeof(double) * nc) : 0;                       // bsrc
    const size_t ld = (size_t)plane_ld(b);
    size_t fac = (mixed ? align16(sizeof(double) * nc) * 3 : 0) + align16(tsz * (size_t)b * ld) +
                 align16(tsz * ld) + align16(tsz * (size_t)b) + 16;
    size_t sol = align16(tsz * 2 * stage_cap((int)crw, b));
    if (mixed) s += align16(tsz * NR3 * nc) + align16(tsz * NR3 * (size_t)b);  // W vb persistent
    else sol += align16(tsz * NR3 * nc) + align16(tsz * NR3 * (size_t)b);      // W vb in the solve overlay
    s += fac > sol ? fac : sol;
    s += align16(sizeof(double) * NR3 * 6 * 3 * 2) + 32 + 64 + 16;
    return s + 64;
}

template <typename T>
struct Carve3 {
    Ops3 O;
    T* c2s;
    double* lam;
    double* bsrc;
    T *Sb, *rowbuf, *colbuf, *ipb;   // factor phase
    double* X;                       // solve phase (mixed: global scratch)
    T *W, *vb, *cbuf, *red;
    uint64_t* bar;
    double* macc;
    int* flags;
    unsigned int* nrm;
    size_t end;   // bytes of shared memory the layout takes
};

template <typename T>
__device__ Carve3<T> carve3(unsigned char* base, const Box3& B, bool stored_rhs, double* xglobal) {
    constexpr bool mixed = std::is_same<T, float>::value;
    Carve3<T> C;
    const size_t nc = B.nc, b = B.b;
    const size_t per = B.soff[6];
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
    C.O.cd = (double*)take(sizeof(double) * nc);
    if (mixed) {
        C.O.dsc = (double*)take(sizeof(double) * nc);
        C.c2s = (T*)take(sizeof(T) * nc);
    } else {
        C.O.dsc = nullptr;
        C.O.c0 = (double*)take(sizeof(double) * nc);
        C.O.c1 = (double*)take(sizeof(double) * nc);
        C.O.c2 = (double*)take(sizeof(double) * nc);
        C.c2s = (T*)C.O.c2;
    }
    C.O.nb = (unsigned char*)take(nc);
    C.O.bT = (double*)take(sizeof(double) * per);
    C.O.bB = (double*)take(sizeof(double) * per);
    C.lam = (double*)take(sizeof(double) * per);
    C.bsrc = stored_rhs ? (double*)take(sizeof(double) * nc) : nullptr;
    if (mixed) {
        C.W = (T*)take(sizeof(T) * NR3 * nc);
        C.vb = (T*)take(sizeof(T) * NR3 * b);
        C.X = xglobal;
    }
    const size_t u0 = o;
    if (mixed) {
        C.O.c0 = (double*)take(sizeof(double) * nc);
        C.O.c1 = (double*)take(sizeof(double) * nc);
        C.O.c2 = (double*)take(sizeof(double) * nc);
    }
    const size_t ld = (size_t)plane_ld((int)b);
    C.Sb = (T*)take(sizeof(T) * b * ld);
    C.rowbuf = (T*)take(sizeof(T) * ld);
    C.colbuf = (T*)take(sizeof(T) * b);
    C.ipb = (T*)take(16);
    const size_t u1 = o;
    o = u0;
    C.cbuf = (T*)take(sizeof(T) * 2 * stage_cap(B.crows, (int)b));
    if (!mixed) {
        C.W = (T*)take(sizeof(T) * NR3 * nc);
        C.X = xglobal;
        C.vb = (T*)take(sizeof(T) * NR3 * b);
    }
    if (o < u1) o = u1;
    C.red = C.vb;   // the sweeps' partial sums reuse the sweep input (NR3 * b >= NR3 * rows)
    C.macc = (double*)take(sizeof(double) * NR3 * 6 * 3 * 2);
    C.flags = (int*)take(32);
    C.nrm = (unsigned int*)take(64);
    C.bar = (uint64_t*)take(16);
    C.end = o;
    return C;
}

}  // namespace

// ---------------------------------------------------------------------------
// Steps 1, 2, 4 and 6 of Algorithm 1 for 3D subdomains (one CTA per job).
// The factor goes to the job's slot: the kept smoothing factor (basis job
// with alpha_basis == alpha_smooth, or the Step 6 job), or scratch.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(T3) k_local3d(DevPtrs P, MethodDev Mth, const Job* jobs) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool mixed = std::is_same<T, float>::value;
    const Job job = jobs[blockIdx.x];
    const SubDev sd = P.sub[job.item];
    const MemberDev& md = P.mem[sd.member];
    __shared__ Box3 B;
    if (threadIdx.x == 0) {
        if (job.type == JOB_PART) setup_box3(B, md, sd.lo, sd.hi, Mth.alpha_b);
        else setup_box3(B, md, sd.loh, sd.hih, job.type == JOB_SFACT ? Mth.alpha_s : Mth.alpha_b);
    }
    if (threadIdx.x == 0) B.crows = stream_rows(B.b, mixed);
    __syncthreads();
    const bool part = job.type == JOB_PART;
    Carve3<T> C = carve3<T>(smem, B, part, P.xs + (size_t)blockIdx.x * P.xs_stride);
    if (!mrcm_check(P.status, C.end <= mrcm_dyn_smem_bytes(), 6, (long long)C.end)) return;   // uniform
    uint32_t par[2] = {0u, 0u};
    if (threadIdx.x == 0) {
        C.flags[0] = 0;
        C.flags[1] = 0;
        C.flags[2] = 0;
        mbar_init(&C.bar[0], 1);
        mbar_init(&C.bar[1], 1);
    }
    build_ops3(B, md, P, C.O, mixed);
    if (mixed)
        for (int t = threadIdx.x; t < B.nc; t += blockDim.x)
            C.c2s[t] = (T)(C.O.c2[t] * C.O.dsc[t] * ((C.O.nb[t] & 32) ? C.O.dsc[t + B.b] : 0.0));
    __syncthreads();
    T* F;
    if (part) F = (T*)P.fac_part + (size_t)job.item * P.part_stride;
    else if (job.type == JOB_SFACT || Mth.same_alpha) F = (T*)P.fac + (size_t)job.item * P.fac_stride;
    else F = (T*)P.fac_aux + (size_t)job.item * P.fac_stride;
    factor3<T>(B, C.O, C.c2s, F, C.Sb, C.rowbuf, C.colbuf, C.ipb, &C.flags[0], mixed);
    if (!part && (job.type == JOB_SFACT || Mth.same_alpha)) {
        double* dd = P.dsc + (size_t)job.item * P.dsc_stride;
        for (int t = threadIdx.x; t < B.nc; t += blockDim.x) dd[t] = mixed ? C.O.dsc[t] : 1.0;
    }
    if (C.flags[0] && threadIdx.x == 0) {
        atomicOr(&P.status[0], ST_NOT_SPD);
        atomicExch(&P.status[2], job.item);
    }
    // with the particular problem on hat-Omega_i (a variant) it is the basis
    // job's last right-hand side, k = nbasis, its vector kept in global memory
    const bool hat_part = job.type == JOB_BASIS && Mth.part_hat;
    const int nrhs = job.type == JOB_BASIS ? sd.nbasis + (hat_part ? 1 : 0) : (part ? 1 : 0);
    if (nrhs == 0) return;

    const int npsi = Mth.npsi;
    const double vol = md.h[0] * md.h[1] * md.h[2];
    const double* fm = P.f + md.cell_off;
    double* bsg = hat_part ? P.bsrc + (size_t)job.item * P.dsc_stride : nullptr;
    if (part || hat_part) {
        double* bs = part ? C.bsrc : bsg;
        for (int t = threadIdx.x; t < B.nc; t += blockDim.x) bs[t] = source_rhs3(B, C.O, md, fm, nullptr, t);
        __syncthreads();
    }
    int nI[3], off[3];
    for (int a = 0; a < 3; ++a) {
        nI[a] = sd.hi[a] - sd.lo[a];
        off[a] = sd.lo[a] - B.lo[a];
    }
    const int nIc = nI[0] * nI[1] * nI[2];
    int maxit = 0, nsolve = 0;
    for (int k0 = 0; k0 < nrhs; k0 += NR3) {
        const int nr = min(NR3, nrhs - k0);
        int it;
        RhsBasis3 rb;
        rb.B = &B;
        rb.bT = C.O.bT;
        rb.bs = bsg;
        if (!part) {
            for (int q = 0; q < nr; ++q) {
                const int k = k0 + q;
                int qq = k / npsi;
                rb.mk[q] = k % npsi;
                rb.sk[q] = k >= sd.nbasis ? -1 : 0;
                if (k >= sd.nbasis) continue;
                for (int sid = 0; sid < 6; ++sid)
                    if (sd.side_mask & (1 << sid)) {
                        if (qq == 0) { rb.sk[q] = sid; break; }
                        --qq;
                    }
            }
            it = solve3<T>(B, md, P.Tf + md.cell_off * 3, C.O, F, C.c2s, C.X, C.W, C.vb, C.cbuf, C.red, C.bar, par, C.nrm, nr, rb, Mth.ir_tol,
                           Mth.max_ir, &C.flags[1], &C.flags[2]);
        } else {
            RhsStored3 rs{C.bsrc};
            it = solve3<T>(B, md, P.Tf + md.cell_off * 3, C.O, F, C.c2s, C.X, C.W, C.vb, C.cbuf, C.red, C.bar, par, C.nrm, nr, rs, Mth.ir_tol,
                           Mth.max_ir, &C.flags[1], &C.flags[2]);
        }
        maxit = max(maxit, it);
        nsolve += it * nr;
        __syncthreads();
        // ---- outputs: restriction to Omega_i, Gamma_i velocities and moments ----
        for (int t = threadIdx.x; t < NR3 * 6 * 3 * 2; t += blockDim.x) C.macc[t] = 0.0;
        for (int q = 0; q < nr; ++q) {
            const double* x = C.X + (size_t)q * B.nc;
            const bool pq = part || k0 + q >= sd.nbasis;   // the particular problem
            double* psi_out = pq ? P.pbar + (size_t)job.item * P.ncell_i_max
                                 : P.Psi + ((size_t)job.item * P.nbasis_max + k0 + q) * P.ncell_i_max;
            for (int ci = threadIdx.x; ci < nIc; ci += blockDim.x) {
                int c[3];
                c[0] = ci % nI[0] + off[0];
                c[1] = (ci / nI[0]) % nI[1] + off[1];
                c[2] = ci / (nI[0] * nI[1]) + off[2];
                psi_out[ci] = x[bidx(B, c)];
            }
        }
        __syncthreads();
        for (int q = 0; q < nr; ++q) {
            const double* x = C.X + (size_t)q * B.nc;
            const int k = k0 + q;
            const bool pq = part || k >= sd.nbasis;
            for (int sid = 0; sid < 6; ++sid) {
                if (!(sd.side_mask & (1 << sid))) continue;
                const int a = sid >> 1;
                const int ts = B.ts[sid], tt = B.tt[sid];
                const int ls = nI[ts], lt = nI[tt];
                const double area = vol / md.h[a];
                const double rarea = 1.0 / area;
                double* ug = pq ? P.ubg + ((size_t)job.item * MRCM_MAXSIDE + sid) * P.side_max
                                : P.Ug + (((size_t)job.item * P.nbasis_max + k) * MRCM_MAXSIDE + sid) * P.side_max;
                for (int e = threadIdx.x; e < ls * lt; e += blockDim.x) {
                    int c[3];
                    c[a] = (sid & 1) ? off[a] + nI[a] - 1 : off[a];
                    c[ts] = off[ts] + e % ls;
                    c[tt] = off[tt] + e / ls;
                    const int tL = bidx(B, c);
                    const double pL = x[tL];
                    const long long gL = gidx(B, md, c);
                    const double hkL = P.hk[(md.cell_off + gL) * 3 + a];
                    int cn[3] = {c[0], c[1], c[2]};
                    cn[a] += (sid & 1) ? 1 : -1;
                    const bool inner = cn[a] >= 0 && cn[a] < B.n[a];
                    double uo, pi;
                    if (inner) {
                        const long long gf = (sid & 1) ? gL : gL - gstride(md, a);
                        const double Tf = P.Tf[(md.cell_off + gf) * 3 + a];
                        uo = Tf * (pL - x[bidx(B, cn)]) * rarea;
                        pi = pL - uo * hkL;
                    } else {
                        const int eb = B.soff[sid] + side_e(B, sid, c);
                        double lam = 0.0;
                        if (!pq && sid == rb.sk[q])
                            lam = psi3(rb.mk[q], c[ts], B.n[ts], c[tt], B.n[tt]);
                        uo = C.O.bT[eb] * (pL - lam) * rarea;
                        pi = part ? C.O.bB[eb] * uo : pL - uo * hkL;
                    }
                    ug[e] = uo;
                    const int cs = e % ls, ct = e / ls;
                    for (int m = 0; m < npsi; ++m) {
                        const double ps = psi3(m, cs, ls, ct, lt);
                        atomicAdd(&C.macc[((q * 6 + sid) * 3 + m) * 2 + 0], ps * uo * area);
                        atomicAdd(&C.macc[((q * 6 + sid) * 3 + m) * 2 + 1], area * ps * pi);
                    }
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nr * 6 * npsi * 2; t += blockDim.x) {
            const int w = t & 1, m = (t >> 1) % npsi, sid = ((t >> 1) / npsi) % 6, q = (t >> 1) / (npsi * 6);
            if (!(sd.side_mask & (1 << sid))) continue;
            const int slot = (part || k0 + q >= sd.nbasis) ? P.nbasis_max : k0 + q;
            P.mom[((((size_t)job.item * (P.nbasis_max + 1) + slot) * MRCM_MAXSIDE + sid) * npsi + m) * 2 + w] =
                C.macc[((q * 6 + sid) * 3 + m) * 2 + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(&P.status[1], maxit);
        atomicAdd(&P.status[3], nsolve);
        if (C.flags[1]) atomicOr(&P.status[0], ST_NO_CONV);
        if (C.flags[2]) atomicOr(&P.status[0], ST_BAD);
    }
}

// ---------------------------------------------------------------------------
// Step 7 in 3D: one colour phase of a smoothing step (Sec. 3, Eqs.
// (sm_1)-(sm_2)), one CTA per subdomain of the colour, kept factor read from
// global memory.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(T3) k_smooth3d(DevPtrs P, MethodDev Mth, const int* items) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool mixed = std::is_same<T, float>::value;
    const int item = items[blockIdx.x];
    const SubDev sd = P.sub[item];
    const MemberDev& md = P.mem[sd.member];
    __shared__ Box3 B;
    if (threadIdx.x == 0) {
        setup_box3(B, md, sd.loh, sd.hih, Mth.alpha_s);
        B.crows = stream_rows(B.b, mixed);
    }
    __syncthreads();
    Carve3<T> C = carve3<T>(smem, B, true, P.xs + (size_t)blockIdx.x * P.xs_stride);
    if (!mrcm_check(P.status, C.end <= mrcm_dyn_smem_bytes(), 6, (long long)C.end)) return;   // uniform
    uint32_t par[2] = {0u, 0u};
    if (threadIdx.x == 0) {
        C.flags[0] = 0;
        C.flags[1] = 0;
        C.flags[2] = 0;
        mbar_init(&C.bar[0], 1);
        mbar_init(&C.bar[1], 1);
    }
    build_ops3(B, md, P, C.O, false);
    const double* dd = P.dsc + (size_t)item * P.dsc_stride;
    if (mixed) {
        for (int t = threadIdx.x; t < B.nc; t += blockDim.x) C.O.dsc[t] = dd[t];
        __syncthreads();
        for (int t = threadIdx.x; t < B.nc; t += blockDim.x)
            C.c2s[t] = (T)(C.O.c2[t] * C.O.dsc[t] * ((C.O.nb[t] & 32) ? C.O.dsc[t + B.b] : 0.0));
    }
    // Robin data from the current solution: lambda = -beta u.n + pi (n outward of hat-Omega_i)
    const double* pst = P.p + md.cell_off;
    const double* ust = P.u + md.cell_off * 6;
    for (int sid = 0; sid < 6; ++sid) {
        if (B.kind[sid] != 2) continue;
        const int a = sid >> 1;
        const int ls = B.n[B.ts[sid]];
        const int faces = B.soff[sid + 1] - B.soff[sid];
        for (int e = threadIdx.x; e < faces; e += blockDim.x) {
            int c[3];
            c[a] = (sid & 1) ? B.n[a] - 1 : 0;
            c[B.ts[sid]] = e % ls;
            c[B.tt[sid]] = e / ls;
            const long long g = gidx(B, md, c);
            const double un = ust[g * 6 + sid];
            const double pi = pst[g] - un * P.hk[(md.cell_off + g) * 3 + a];
            C.lam[B.soff[sid] + e] = -C.O.bB[B.soff[sid] + e] * un + pi;
        }
    }
    __syncthreads();
    const double* fm = P.f + md.cell_off;
    for (int t = threadIdx.x; t < B.nc; t += blockDim.x) C.bsrc[t] = source_rhs3(B, C.O, md, fm, C.lam, t);
    __syncthreads();
    const T* F = (const T*)P.fac + (size_t)item * P.fac_stride;
    RhsStored3 rs{C.bsrc};
    const int it = solve3<T>(B, md, P.Tf + md.cell_off * 3, C.O, F, C.c2s, C.X, C.W, C.vb, C.cbuf, C.red, C.bar, par, C.nrm, 1, rs, Mth.ir_tol,
                             Mth.max_ir, &C.flags[0], &C.flags[2]);
    __syncthreads();
    // overwrite (u, p) on Omega_i with the restriction
    int nI[3], off[3];
    for (int a = 0; a < 3; ++a) {
        nI[a] = sd.hi[a] - sd.lo[a];
        off[a] = sd.lo[a] - B.lo[a];
    }
    const int nIc = nI[0] * nI[1] * nI[2];
    double* pw = P.p + md.cell_off;
    double* uw = P.u + md.cell_off * 6;
    const double vol = md.h[0] * md.h[1] * md.h[2];
    const double* x = C.X;
    for (int ci = threadIdx.x; ci < nIc; ci += blockDim.x) {
        int c[3];
        c[0] = ci % nI[0] + off[0];
        c[1] = (ci / nI[0]) % nI[1] + off[1];
        c[2] = ci / (nI[0] * nI[1]) + off[2];
        const int t = bidx(B, c);
        const long long g = gidx(B, md, c);
        if (!mrcm_check(P.status, g >= 0 && g < (long long)md.n[0] * md.n[1] * md.n[2], 7, g)) continue;
        const double pc = x[t];
        pw[g] = pc;
        for (int sid = 0; sid < 6; ++sid) {
            const int a = sid >> 1;
            const double rarea = md.h[a] / vol;
            int cn[3] = {c[0], c[1], c[2]};
            cn[a] += (sid & 1) ? 1 : -1;
            double uo;
            if (cn[a] >= 0 && cn[a] < B.n[a]) {
                const long long gf = (sid & 1) ? g : g - gstride(md, a);
                uo = P.Tf[(md.cell_off + gf) * 3 + a] * (pc - x[bidx(B, cn)]) * rarea;
            } else {
                const int eb = B.soff[sid] + side_e(B, sid, c);
                if (B.kind[sid] == 2) uo = C.O.bT[eb] * (pc - C.lam[eb]) * rarea;
                else if (B.kind[sid] == 1) uo = C.O.bT[eb] * (pc - B.val[sid]) * rarea;
                else uo = B.val[sid];
            }
            uw[g * 6 + sid] = uo;
        }
    }
    if (threadIdx.x == 0) {
        atomicMax(&P.status[1], it);
        atomicAdd(&P.status[3], it);
        if (C.flags[0]) atomicOr(&P.status[0], ST_NO_CONV);
        if (C.flags[2]) atomicOr(&P.status[0], ST_BAD);
    }
}

// ---------------------------------------------------------------------------
// Superposition in 3D (Eqs. (addu), (addp), (uhatphat)): p = pbar + sum_k
// X_k Psi_k on Omega_i; Gamma_i velocities ubar + sum_k X_k U_k; interior
// faces from the assembled pressure; physical faces from the data.
// ---------------------------------------------------------------------------
__global__ void k_assemble3d(DevPtrs P, const double* __restrict__ X) {
    extern __shared__ double ps3[];
    const int item = blockIdx.x;
    const SubDev sd = P.sub[item];
    const MemberDev& md = P.mem[sd.member];
    int nI[3];
    for (int a = 0; a < 3; ++a) nI[a] = sd.hi[a] - sd.lo[a];
    const int n = nI[0] * nI[1] * nI[2];
    const double* xs = X + sd.col0;
    const double* Psi = P.Psi + (size_t)item * P.nbasis_max * P.ncell_i_max;
    const double* pb = P.pbar + (size_t)item * P.ncell_i_max;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double v = pb[c];
        for (int k = 0; k < sd.nbasis; ++k) v += xs[k] * Psi[(size_t)k * P.ncell_i_max + c];
        ps3[c] = v;
    }
    __syncthreads();
    const double* Tf = P.Tf + md.cell_off * 3;
    const double* hk = P.hk + md.cell_off * 3;
    double* pw = P.p + md.cell_off;
    double* uw = P.u + md.cell_off * 6;
    const double vol = md.h[0] * md.h[1] * md.h[2];
    const int cst[3] = {1, nI[0], nI[0] * nI[1]};
    for (int ci = threadIdx.x; ci < n; ci += blockDim.x) {
        int c[3];
        c[0] = ci % nI[0];
        c[1] = (ci / nI[0]) % nI[1];
        c[2] = ci / (nI[0] * nI[1]);
        const long long g = (sd.lo[0] + c[0]) + (long long)md.n[0] * ((sd.lo[1] + c[1]) + (long long)md.n[1] * (sd.lo[2] + c[2]));
        if (!mrcm_check(P.status, g >= 0 && g < (long long)md.n[0] * md.n[1] * md.n[2], 7, g)) continue;
        const double pc = ps3[ci];
        pw[g] = pc;
        for (int sid = 0; sid < 6; ++sid) {
            const int a = sid >> 1;
            const bool hi = sid & 1;
            const bool edge = hi ? (c[a] == nI[a] - 1) : (c[a] == 0);
            const double rarea = md.h[a] / vol;
            const long long gs = a == 0 ? 1LL : a == 1 ? (long long)md.n[0] : (long long)md.n[0] * md.n[1];
            double uo;
            if (!edge) {
                const int cn = ci + (hi ? cst[a] : -cst[a]);
                const long long gf = hi ? g : g - gs;
                uo = Tf[gf * 3 + a] * (pc - ps3[cn]) * rarea;
            } else if (sd.side_mask & (1 << sid)) {
                const int ts = a == 0 ? 1 : 0, tt = a == 2 ? 1 : 2;
                const int e = c[ts] + nI[ts] * c[tt];
                double v = P.ubg[((size_t)item * MRCM_MAXSIDE + sid) * P.side_max + e];
                for (int k = 0; k < sd.nbasis; ++k)
                    v += xs[k] * P.Ug[(((size_t)item * P.nbasis_max + k) * MRCM_MAXSIDE + sid) * P.side_max + e];
                uo = v;
            } else if (md.bc_kind[sid] == 1) {
                uo = (pc - md.bc_val[sid]) / (hk[g * 3 + a]) ;   // T / a = 1 / hk
            } else {
                uo = md.bc_val[sid];
            }
            uw[g * 6 + sid] = uo;
        }
    }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
size_t local3d_smem(int prec, int nx, int ny, int nz, bool part) {
    return carve3_bytes(prec == 0 ? 8 : 4, nx, ny, nz, part);
}

size_t smooth3d_smem(int prec, int nx, int ny, int nz) { return carve3_bytes(prec == 0 ? 8 : 4, nx, ny, nz, true); }

// entries of one box factor (n_a2 planes of b x b)
// The bulk copies of the sweeps need 16-byte aligned sources, destinations
// and sizes: plane strides, chunk offsets and staging capacities of a box.
bool stage3_aligned(int prec, int nx, int ny, int nz) {
    int b, npl;
    box3_dims(nx, ny, nz, &b, &npl);
    const size_t tsz = prec == 0 ? sizeof(double) : sizeof(float);
    const int rows = stream_rows(b, prec != 0);
    const size_t cap = stage_cap(rows, b);
    const int nch = (b + rows - 1) / rows;
    if ((plane_stride(b) * tsz) % 16 || (cap * tsz) % 16) return false;
    if (nch > 1 && ((size_t)rows * b * tsz) % 16) return false;          // chunk starts
    const size_t c0 = (size_t)(nch - 1) * rows;                            // last chunk
    const size_t last = (((size_t)b - c0) * b * tsz + 15) & ~size_t(15);   // its rounded size
    return last <= cap * tsz && c0 * b * tsz + last <= plane_stride(b) * tsz;
}

size_t factor3_entries(int nx, int ny, int nz) {
    int b, npl;
    box3_dims(nx, ny, nz, &b, &npl);
    return plane_stride(b) * npl;
}

template <typename T>
static cudaError_t launch_local3d_t(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs, size_t smem,
                                    cudaStream_t s) {
    static size_t cur = 0;
    if (smem > cur) {
        cudaError_t e = cudaFuncSetAttribute(k_local3d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cur = smem;
    }
    k_local3d<T><<<njobs, T3, smem, s>>>(P, M, jobs);
    return cudaGetLastError();
}

cudaError_t launch_local3d(const DevPtrs& P, const MethodDev& M, const Job* jobs, int njobs, size_t smem,
                           cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    return M.prec == 0 ? launch_local3d_t<double>(P, M, jobs, njobs, smem, s)
                       : launch_local3d_t<float>(P, M, jobs, njobs, smem, s);
}

template <typename T>
static cudaError_t launch_smooth3d_t(const DevPtrs& P, const MethodDev& M, const int* items, int nitems, size_t smem,
                                     cudaStream_t s) {
    static size_t cur = 0;
    if (smem > cur) {
        cudaError_t e = cudaFuncSetAttribute(k_smooth3d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cur = smem;
    }
    k_smooth3d<T><<<nitems, T3, smem, s>>>(P, M, items);
    return cudaGetLastError();
}

cudaError_t launch_smooth3d(const DevPtrs& P, const MethodDev& M, const int* items, int nitems, size_t smem,
                            cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    return M.prec == 0 ? launch_smooth3d_t<double>(P, M, items, nitems, smem, s)
                       : launch_smooth3d_t<float>(P, M, items, nitems, smem, s);
}

cudaError_t launch_assemble3d(const DevPtrs& P, const double* X, int nitems, int ncell_i_max, cudaStream_t s) {
    k_assemble3d<<<nitems, 256, sizeof(double) * ncell_i_max, s>>>(P, X);
    return cudaGetLastError();
}
