// Vector kernels of the interface Krylov fallback (FP64 GMRES on the
// interface system of Eqs. (int_ujump)-(int_pjump), right-preconditioned by
// the FP32 block-cyclic reduction; the driver is krylov_interface in api.cu).
#include "mrcm_internal.cuh"

// Used only when the refinement stalls.  The preconditioner reads its input
// through the row scaling into bq and returns the column-scaled result, as
// one refinement step does.

__global__ void k_kry_to_bq(IfPtrs I, const double* v, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) I.bq[c] = (float)(I.R[c] * v[c]);
}

__global__ void k_kry_from_bq(IfPtrs I, double* z, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) z[c] = I.Cs[c] * (double)I.bq[c];
}

// y = a x + b y (b = 0: y = a x, whatever y held)
__global__ void k_kry_axpby(double* y, const double* x, double a, double b, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) y[c] = b == 0.0 ? a * x[c] : a * x[c] + b * y[c];
}

// per-block partial sums of a . b (grid-stride, fixed order within a block)
constexpr int KRY_BLOCKS = 120;
constexpr int KRY_MAXV = 32;   // vectors of one projection step at most (the restart length + 1)
__global__ void __launch_bounds__(256) k_kry_dot(const double* a, const double* b, int n, double* part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) acc += a[c] * b[c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

cudaError_t kry_to_bq(const IfPtrs& I, const double* v, int n, cudaStream_t s) {
    k_kry_to_bq<<<(n + 255) / 256, 256, 0, s>>>(I, v, n);
    return cudaGetLastError();
}

cudaError_t kry_from_bq(const IfPtrs& I, double* z, int n, cudaStream_t s) {
    k_kry_from_bq<<<(n + 255) / 256, 256, 0, s>>>(I, z, n);
    return cudaGetLastError();
}

cudaError_t kry_axpby(double* y, const double* x, double a, double b, int n, cudaStream_t s) {
    k_kry_axpby<<<(n + 255) / 256, 256, 0, s>>>(y, x, a, b, n);
    return cudaGetLastError();
}

// part: KRY_BLOCKS doubles of device memory
cudaError_t kry_dot(const double* a, const double* b, int n, double* part, cudaStream_t s) {
    k_kry_dot<<<KRY_BLOCKS, 256, 0, s>>>(a, b, n, part);
    return cudaGetLastError();
}

int kry_blocks() { return KRY_BLOCKS; }

// Block partial sums of v_i . w for the nv vectors v_i = V + i n (classical
// Gram-Schmidt: all projections of one step in one launch): part[i * KRY_BLOCKS + block].
__global__ void __launch_bounds__(256) k_kry_mdot(const double* V, const double* w, int n, int nv, double* part) {
    __shared__ double red[256];
    for (int i = 0; i < nv; ++i) {
        const double* v = V + (size_t)i * n;
        double acc = 0.0;
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) acc += v[c] * w[c];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = 128; o; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)i * gridDim.x + blockIdx.x] = red[0];
        __syncthreads();
    }
}

// w -= sum_i c_i v_i over the nv vectors v_i = V + i n (in increasing i per entry)
struct KryCoef {
    double c[KRY_MAXV];
};
__global__ void k_kry_msub(double* w, const double* V, KryCoef cf, int nv, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double x = w[c];
    for (int i = 0; i < nv; ++i) x -= cf.c[i] * V[(size_t)i * n + c];
    w[c] = x;
}

cudaError_t kry_mdot(const double* V, const double* w, int n, int nv, double* part, cudaStream_t s) {
    k_kry_mdot<<<KRY_BLOCKS, 256, 0, s>>>(V, w, n, nv, part);
    return cudaGetLastError();
}

cudaError_t kry_msub(double* w, const double* V, const double* coef, int nv, int n, cudaStream_t s) {
    if (nv > KRY_MAXV) return cudaErrorInvalidValue;
    KryCoef cf{};
    for (int i = 0; i < nv; ++i) cf.c[i] = coef[i];
    k_kry_msub<<<(n + 255) / 256, 256, 0, s>>>(w, V, cf, nv, n);
    return cudaGetLastError();
}
