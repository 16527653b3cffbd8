// Slab inverses of the interface reduction (Algorithm 1, Step 5: the block
// cyclic reduction needs D_j^-1 of every eliminated slab) by unblocked
// Gauss-Jordan elimination with partial pivoting, the slab held in registers
// across a cluster of CTAs.
//
// The (padded, column-major) NPAD x NPAD slab is split into panels of CB
// consecutive columns; warp w of CTA r in a cluster of CL CTAs holds panel
// r NW + w, rows l + 32 a (a < RA) on lane l, in registers for the whole
// elimination, so no matrix entry moves through memory during it.  Panels
// are eliminated in order, one pivot column at a time:
//   * the warp owning panel P waits for nothing but the records of the
//     panels before it; for each of its columns k it picks the pivot row p
//     (the largest magnitude to 2^-12 relative among the rows not yet used,
//     the first row among equals) by one warp reduction, applies the
//     rank-1 update A_ij -= A_ik A_pj / A_pk to its other columns, sets
//     column k to -A_ik / A_pk (1 in row p, see below) and writes the
//     column's values with the entry of row p zeroed (the multipliers), p
//     and the pivot into the panel's record in its CTA's shared memory; the
//     finished record goes to every other CTA of the cluster by one bulk
//     copy each (completing an mbarrier there by its bytes) and is released
//     in its own CTA by one arrival;
//   * every other warp waits for the record and applies the panel's CB
//     rank-1 updates to its own columns in turn, each taking the pivot row's
//     current values on its columns from the lane holding row p (selected
//     from that lane's register slots by a binary tree, since the slot is
//     only known at run time, then broadcast by a shuffle).
// The pivot search thus never leaves a warp, and the warps synchronise once
// per panel instead of once per column.  Row p is not rescaled by 1 / A_pk
// in its step: each stored row carries the factor c_i (1 until the row
// becomes a pivot, then its pivot value), so the record's entries are the
// multipliers themselves and the pivot row needs no write to a register slot
// chosen at run time.  The stored rows are divided by c_i at the end.  After
// the last step the storage holds (P A)^-1 for the row permutation P of the
// pivots.  The slab eliminated is D^T, and its inverse is written out
// transposed: D^-1 = ((D^T)^-1)^T, entry (i, j) of the storage going to row
// pivrow[j] of column pinv[i].  Gauss-Jordan's inverse has the smaller
// residual on one side; eliminating D^T puts it on the side the reduction
// uses (the FP64 refinement of the interface solve needs 5 steps on the
// 512x512 channel workload instead of 9 when D itself is eliminated, the
// same as with the LU).  The arithmetic is that of unblocked Gauss-Jordan
// elimination (n^3 multiply-adds for n unknowns), in FP32.
//
// Records live in a ring of R slots.  A cluster barrier every G panels
// bounds how far a producer can run ahead (R = 2 G: a slot is rewritten only
// after every CTA has read it) and lets each CTA re-arm a slot right after
// reading it.  Every wait on a record is bounded; a wait that runs out marks
// the launch (ST_BAD) and the kernel runs to its end without further waits.
#include "mrcm_internal.cuh"

#include <cuda_runtime.h>

#include <utility>

namespace {

constexpr unsigned GR_FULL = 0xffffffffu;
constexpr long long GR_WAIT_LIMIT = 1LL << 24;   // polls of one record's mbarrier before giving up

__device__ __forceinline__ unsigned gr_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned gr_mapa(unsigned addr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ unsigned gr_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void gr_arm(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool gr_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void gr_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 1 / x from the hardware approximation and one Newton-Raphson step
// (e = 1 - x r, r + r e), within an ulp or so of the rounded reciprocal
__device__ __forceinline__ float gr_rcp(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = fmaf(-x, r, 1.f);
    return fmaf(r, e, r);
}

__device__ __forceinline__ void gr_release(int* flag, int v) {
    asm volatile("st.release.cta.shared::cta.s32 [%0], %1;" ::"r"(gr_smem(flag)), "r"(v) : "memory");
}

__device__ __forceinline__ int gr_acquire(const int* flag) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(gr_smem(flag)) : "memory");
    return v;
}

__device__ __forceinline__ void gr_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename F, int... Is>
__device__ __forceinline__ void gr_static_for(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}

template <int NPAD, int CL, int NW>
struct GrShape {
    static constexpr int NT = 32 * NW;              // threads per CTA
    static constexpr int CB = NPAD / (CL * NW);     // columns per warp = panel width
    static constexpr int CW = NW * CB;              // columns per CTA
    static constexpr int RA = NPAD / 32;            // rows per lane
    static constexpr int HDR = 4 * CB;              // record header: (p, pivot, 1 / pivot, 0) per column
    static constexpr int REC = CB * NPAD + HDR;     // floats per record
    static_assert(RA % 4 == 0 && (RA < 8 || RA % 8 == 0) && RA <= 32 && CB % 4 == 0 && CB * NW * CL == NPAD,
                  "unsupported slab inverse shape");
    static constexpr int G = NPAD >= 768 ? 2 : NPAD >= 512 ? 4 : 8;   // panels between cluster barriers
    static constexpr int R = 2 * G;                  // record slots (one panel each)
    static constexpr size_t smem() { return sizeof(float) * ((size_t)R * REC + (size_t)NW * NPAD * CB); }
};

template <int NPAD, int CL, int NW>
__global__ void __launch_bounds__(32 * NW, 1) k_gjr_inverse(IfPtrs I, const ElimDev* el, int nel, int* status) {
    using Sh = GrShape<NPAD, CL, NW>;
    constexpr int CB = Sh::CB, CW = Sh::CW, RA = Sh::RA, REC = Sh::REC, G = Sh::G, R = Sh::R;
    constexpr unsigned BYTES = 4u * REC;   // bytes of one record in every CTA
    extern __shared__ __align__(16) float gr_dyn[];
    float* recs = gr_dyn;                  // [R][REC]
    float* tiles = recs + R * REC;         // [warp][NPAD][CB]
    __shared__ __align__(8) unsigned long long bars[R];
    __shared__ int colready[R];            // columns of a slot's record written so far (P CB + c + 1)
    __shared__ int pivrow[NPAD];           // pivot row of every step
    __shared__ float pivval[NPAD];         // its pivot
    __shared__ int pinv[NPAD];             // step at which each row was the pivot
    __shared__ float rsc[NPAD];            // 1 / c_i

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned rank = gr_rank();
    const int e = blockIdx.x / CL;
    if (e >= nel) return;   // the grid holds whole clusters only; uniform per cluster
    const SlabDev S = I.slabs[el[e].j];
    const int n = S.n, np = I.npad;
    const int npan = (n + CB - 1) / CB;    // panels holding a column below n
    const float* A = I.D + S.offD;
    float* Ainv = I.Dinv + S.offD;

    // the transposed slab: entry (i, j) of D^T is A[i np + j] in D's
    // column-major storage, so a lane's CB consecutive columns of row i are
    // contiguous (np and the warp's first column are multiples of 4)
    float V[RA][CB];
    {
        const int j0 = CW * (int)rank + CB * warp;
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int i = lane + 32 * a;
#pragma unroll
            for (int q = 0; q < CB / 4; ++q) {
                const int j = j0 + 4 * q;
                float4 t;
                if (i < np && j < np) {
                    t = __ldcg(reinterpret_cast<const float4*>(A + (size_t)i * np + j));
                } else {
                    t.x = i == j ? 1.f : 0.f;
                    t.y = i == j + 1 ? 1.f : 0.f;
                    t.z = i == j + 2 ? 1.f : 0.f;
                    t.w = i == j + 3 ? 1.f : 0.f;
                }
                V[a][4 * q] = t.x;
                V[a][4 * q + 1] = t.y;
                V[a][4 * q + 2] = t.z;
                V[a][4 * q + 3] = t.w;
            }
        }
    }
    const unsigned rbase = gr_smem(recs), bbase = gr_smem(bars);
    if (tid == 0) {
        for (int q = 0; q < R; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bbase + 8u * (unsigned)q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // a record from another CTA completes the slot's phase by its bytes
        // (armed here); a record of this CTA by its producer's arrival
        for (int q = 0; q < R && q < npan; ++q)
            if (q / NW != (int)rank) gr_arm(bbase + 8u * (unsigned)q, BYTES);
    }
    for (int i = tid; i < NPAD; i += Sh::NT) {
        pivrow[i] = i;
        pivval[i] = 1.f;
    }
    if (tid < R) colready[tid] = 0;
    gr_cluster_sync();

    unsigned usedm = 0u;   // bit a: row lane + 32 a has been a pivot
    unsigned rowok = 0u;   // bit a: row lane + 32 a is below n
#pragma unroll
    for (int a = 0; a < RA; ++a) rowok |= (lane + 32 * a < n ? 1u : 0u) << a;
    bool timed_out = false, singular = false;
    float* tile = tiles + (size_t)warp * NPAD * CB;   // this warp's columns at the start of a panel, by row
    // multiplier of panel column c at row i in a record
    auto mult = [&](const float* rc, int c, int i) { return rc[c * NPAD + (i & 31) * RA + (i >> 5)]; };

#pragma unroll 1
    for (int P = 0; P < npan; ++P) {
        if (P > 0 && P % G == 0) {
            __syncwarp();
            gr_cluster_sync();
        }
        const int slot = P % R;
        const unsigned bar = bbase + 8u * (unsigned)slot;
        float* rc = recs + slot * REC;
        const bool mine = P / NW == (int)rank && P % NW == warp;
        // the owner of the next panel, when both panels are this CTA's, takes
        // the record column by column as it is written (its update of the
        // last column is then all that stands between the two panels)
        const bool follow = !mine && P / NW == (int)rank && (P + 1) / NW == (int)rank && (P + 1) % NW == warp;
        if (!mine && !follow && !timed_out) {
            long long it = 0;
            while (!gr_try(bar, (unsigned)(P / R) & 1u))
                if (++it > GR_WAIT_LIMIT) {
                    timed_out = true;
                    break;
                }
        }
        // the panel's pivot rows are looked up in this copy: the values a
        // pivot row had on this warp's columns when the panel began
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int q = 0; q < CB / 4; ++q)
                *reinterpret_cast<float4*>(tile + (lane + 32 * a) * CB + 4 * q) =
                    make_float4(V[a][4 * q], V[a][4 * q + 1], V[a][4 * q + 2], V[a][4 * q + 3]);
        __syncwarp();
        // u[c][b]: row p_c of column b just before step c, divided by the pivot
        float u[CB][CB];
        if (mine) {
            // ---- this warp's panel: CB pivots, each column recorded as it is eliminated
            float ipc[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const int k = P * CB + c;
                ipc[c] = 1.f;
#pragma unroll
                for (int b = 0; b < CB; ++b) u[c][b] = 0.f;
                if (k >= n) continue;   // uniform; the record's entries for k are never read
                float col[RA];
#pragma unroll
                for (int a = 0; a < RA; ++a) col[a] = V[a][c];
                // the pivot among the unused rows below n: the largest magnitude to
                // 2^-12 relative, the first row among equals (keys carry 2047 - row;
                // a candidate's key is at least 1024 since NPAD <= 1024), by a tree
                // over the lane's rows and one warp reduction
                unsigned key = 0u;
                float best = 0.f;
#pragma unroll
                for (int a0 = 0; a0 < RA; a0 += 8) {   // chunks of 8 rows bound the live registers
                    constexpr int KC = RA < 8 ? RA : 8;
                    unsigned kt[KC];
                    float vt[KC];
#pragma unroll
                    for (int t = 0; t < KC; ++t) {
                        const int a = a0 + t;
                        const float v = fabsf(col[a]);
                        const unsigned kb =
                            ((v == v ? __float_as_uint(v) : 0u) & ~0x7ffu) | (0x7ffu - (unsigned)(lane + 32 * a));
                        kt[t] = ((rowok & ~usedm) >> a) & 1u ? kb : 0u;
                        vt[t] = col[a];
                    }
#pragma unroll
                    for (int w = 1; w < KC; w <<= 1)
#pragma unroll
                        for (int t = 0; t + w < KC; t += 2 * w) {
                            const bool hi = kt[t + w] > kt[t];
                            kt[t] = hi ? kt[t + w] : kt[t];
                            vt[t] = hi ? vt[t + w] : vt[t];
                        }
                    const bool hi = kt[0] > key;
                    key = hi ? kt[0] : key;
                    best = hi ? vt[0] : best;
                }
                const unsigned km = __reduce_max_sync(GR_FULL, key);
                const unsigned wl = __ballot_sync(GR_FULL, km != 0u && key == km);
                const int p = km != 0u ? (int)(0x7ffu - (km & 0x7ffu)) : 0;
                float piv = __shfl_sync(GR_FULL, best, wl ? __ffs(wl) - 1 : 0);
                if (km == 0u || piv == 0.f) {
                    singular = true;
                    piv = 1e-30f;
                }
                const float ip = gr_rcp(piv);
                ipc[c] = ip;
#pragma unroll
                for (int a = 0; a < RA; ++a)
                    if (lane + 32 * a == p) col[a] = 0.f;   // no multiplier for the pivot row
#pragma unroll
                for (int q = 0; q < RA / 4; ++q)
                    *reinterpret_cast<float4*>(rc + c * NPAD + lane * RA + 4 * q) =
                        make_float4(col[4 * q], col[4 * q + 1], col[4 * q + 2], col[4 * q + 3]);
                if (lane == 0) {
                    *reinterpret_cast<float4*>(rc + CB * NPAD + 4 * c) = make_float4(__int_as_float(p), piv, ip, 0.f);
                    pivrow[k] = p;
                    pivval[k] = piv;
                }
                __syncwarp();
                if (lane == 0) gr_release(&colready[slot], P * CB + c + 1);   // column c of the record is complete
                // row p on the other columns just before this step, from the panel's
                // start and the multipliers recorded so far: columns not yet pivots
                // start from the copy, pivot columns b < c from their fixed values
                float x[CB];
#pragma unroll
                for (int q = 0; q < CB / 4; ++q) {
                    const float4 t = *reinterpret_cast<const float4*>(tile + p * CB + 4 * q);
                    x[4 * q] = t.x;
                    x[4 * q + 1] = t.y;
                    x[4 * q + 2] = t.z;
                    x[4 * q + 3] = t.w;
                }
#pragma unroll
                for (int b = 0; b < CB; ++b) {
                    if (b == c) continue;
                    float t = b < c ? -mult(rc, b, p) * ipc[b] : x[b];
#pragma unroll
                    for (int c2 = 0; c2 < c; ++c2)
                        if (c2 > b || b > c) t = fmaf(-mult(rc, c2, p), u[c2][b], t);
                    u[c][b] = t * ip;
                }
#pragma unroll
                for (int b = 0; b < CB; ++b)
                    if (b != c)
#pragma unroll
                        for (int a = 0; a < RA; ++a) V[a][b] = fmaf(-col[a], u[c][b], V[a][b]);
                // column k: -A_ik / A_pk, and c_p / A_pk = 1 in the pivot row
#pragma unroll
                for (int a = 0; a < RA; ++a) V[a][c] = (lane + 32 * a == p) ? 1.f : -col[a] * ip;
                if (lane == (p & 31)) usedm |= 1u << (p >> 5);
            }
            // the finished record: one bulk copy into every other CTA (the
            // copy engine reads it after the proxy fence), one arrival here
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                gr_arrive(bar);   // this CTA's warps first: the next panel's owner is most often here
                const unsigned src = rbase + 4u * (unsigned)(slot * REC);
#pragma unroll 1
                for (int r = 0; r < CL; ++r) {
                    if (r == (int)rank) continue;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            gr_mapa(src, (unsigned)r)),
                        "r"(src), "r"(BYTES), "r"(gr_mapa(bar, (unsigned)r))
                        : "memory");
                }
            }
        } else {
            // ---- another warp's panel: its CB rank-1 updates on this warp's
            // columns, the pivot rows' values by the same recurrence
            const bool remote = P / NW != (int)rank;
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const int k = P * CB + c;
#pragma unroll
                for (int b = 0; b < CB; ++b) u[c][b] = 0.f;
                if (k >= n) continue;
                if (follow && !timed_out) {
                    long long it = 0;
                    while (gr_acquire(&colready[slot]) < k + 1)
                        if (++it > GR_WAIT_LIMIT) {
                            timed_out = true;
                            break;
                        }
                }
                const float4 ph = *reinterpret_cast<const float4*>(rc + CB * NPAD + 4 * c);
                const int pr = __float_as_int(ph.x);
                const int p = mrcm_check(status, timed_out || (unsigned)pr < (unsigned)n, 9, pr) && (unsigned)pr < (unsigned)NPAD
                                  ? pr
                                  : 0;   // a record from a run that timed out may hold anything
                const float ip = ph.z;
                float x[CB];
#pragma unroll
                for (int q = 0; q < CB / 4; ++q) {
                    const float4 t = *reinterpret_cast<const float4*>(tile + p * CB + 4 * q);
                    x[4 * q] = t.x;
                    x[4 * q + 1] = t.y;
                    x[4 * q + 2] = t.z;
                    x[4 * q + 3] = t.w;
                }
#pragma unroll
                for (int c2 = 0; c2 < c; ++c2) {
                    const float mc = mult(rc, c2, p);
#pragma unroll
                    for (int b = 0; b < CB; ++b) x[b] = fmaf(-mc, u[c2][b], x[b]);
                }
#pragma unroll
                for (int b = 0; b < CB; ++b) u[c][b] = x[b] * ip;
                if (lane == (p & 31)) usedm |= 1u << (p >> 5);
                if (remote && tid == 0) {
                    pivrow[k] = p;
                    pivval[k] = ph.y;
                }
                // the column's rank-1 update (the order over the panel's columns per entry is kept)
                float m[RA];
#pragma unroll
                for (int q = 0; q < RA / 4; ++q) {
                    const float4 t = *reinterpret_cast<const float4*>(rc + c * NPAD + lane * RA + 4 * q);
                    m[4 * q] = t.x;
                    m[4 * q + 1] = t.y;
                    m[4 * q + 2] = t.z;
                    m[4 * q + 3] = t.w;
                }
#pragma unroll
                for (int b = 0; b < CB; ++b)
#pragma unroll
                    for (int a = 0; a < RA; ++a) V[a][b] = fmaf(-m[a], u[c][b], V[a][b]);
            }
        }
        __syncwarp();   // the copy is rewritten at the next panel
        // re-arm the slot for the record R panels on, once its phase is complete here
        if (tid == 0 && !timed_out && P + R < npan && (P + R) / NW != (int)rank) gr_arm(bar, BYTES);
    }

    __syncthreads();
    for (int i = tid; i < NPAD; i += Sh::NT) {
        pinv[i] = i;
        rsc[i] = 1.f;
    }
    __syncthreads();
    for (int k = tid; k < n; k += Sh::NT) {
        const int i = pivrow[k];
        pinv[i] = k;
        rsc[i] = gr_rcp(pivval[k]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        const int j = CW * (int)rank + CB * warp + b;
        const int cj = j < np ? pivrow[j] : np;   // pivots are rows below n <= np; checked all the same
        if (cj < np) {
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                const int i = lane + 32 * a;
                const int ri = i < np ? pinv[i] : np;
                if (mrcm_check(status, ri < np || i >= np, 10, ri) && ri < np)
                    Ainv[(size_t)ri * np + cj] = V[a][b] * rsc[i];   // (D^T)^-1 transposed
            }
        }
    }
    if (lane == 0 && singular) atomicOr(status, ST_SINGULAR);
    if (lane == 0 && timed_out) atomicOr(status, ST_BAD);
    __syncwarp();
    gr_cluster_sync();   // no CTA leaves while a peer may still address its shared memory
}

template <int NPAD, int CL, int NW>
cudaError_t launch_gjr(const IfPtrs& I, const ElimDev* el, int nel, int* status, cudaStream_t s) {
    using Sh = GrShape<NPAD, CL, NW>;
    const size_t smem = Sh::smem();
    static size_t set_smem = 0;
    if (smem > set_smem) {
        cudaError_t e =
            cudaFuncSetAttribute(k_gjr_inverse<NPAD, CL, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && CL > 8)
            e = cudaFuncSetAttribute(k_gjr_inverse<NPAD, CL, NW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        set_smem = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nel * CL);
    cfg.blockDim = dim3(Sh::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    IfPtrs Ic = I;
    void* args[] = {&Ic, (void*)&el, &nel, &status};
    return cudaLaunchKernelExC(&cfg, (const void*)k_gjr_inverse<NPAD, CL, NW>, args);
}

}  // namespace

// Template slab size of the register-resident Gauss-Jordan inverse for a
// padded slab size, 0 when it has none (slabs above 768 unknowns).
int slab_inverse_gjr_npad(int npad) {
    return npad <= 128 ? 128 : npad <= 256 ? 256 : npad <= 512 ? 512 : npad <= 768 ? 768 : 0;
}

// One elimination level's slab inverses: the larger cluster when all the
// level's clusters fit on the GPU at once (one CTA per SM), else the smaller.
cudaError_t gjr_inverse(const IfPtrs& I, const ElimDev* el, int nel, int* status, cudaStream_t s) {
    if (nel == 0) return cudaSuccess;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // latency-bound levels (few slabs): 8 CTAs of 8 warps per slab (16 of 8
    // for 512 unknowns) when the level's clusters all fit at once; large
    // batches: fewer, wider CTAs per slab (less cluster traffic per column)
    const bool very_few = nel * 16 <= nsm, few = nel * 8 <= nsm;
    switch (slab_inverse_gjr_npad(I.npad)) {
        case 128: return few ? launch_gjr<128, 4, 8>(I, el, nel, status, s) : launch_gjr<128, 2, 16>(I, el, nel, status, s);
        case 256: return few ? launch_gjr<256, 8, 8>(I, el, nel, status, s) : launch_gjr<256, 4, 16>(I, el, nel, status, s);
        case 512: return very_few ? launch_gjr<512, 16, 8>(I, el, nel, status, s) : launch_gjr<512, 8, 16>(I, el, nel, status, s);
        case 768: return launch_gjr<768, 16, 12>(I, el, nel, status, s);   // 16 CTAs of 12 warps
        default: return cudaErrorInvalidValue;
    }
}
