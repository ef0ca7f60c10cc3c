// Allocation-free variant of the refined solve of (I - K) x = s.
//
// Some callers cannot allocate device memory at the moment they need a solve:
// a host program whose device memory is owned by its own pool allocator and
// sized at start-up, or a latency-critical loop in which cudaMalloc / cudaFree
// (which may synchronise the whole device) are not allowed.  This entry point
// serves them: it takes the matrix, the source and the output from the
// caller and keeps its work vectors in a fixed, file-scope device array that
// is part of the library image, so the call itself allocates nothing.
#include <cuda_runtime.h>

#include <cstdint>

#include "tursca.h"

namespace {

// Largest system the scratch array can hold, and its layout.
constexpr int kMaxNodes = 1 << 20;                 // 1,048,576 nodes
constexpr int kPartBlocks = 1024;                  // residual partial sums
constexpr size_t kOffB = 0;                        // float  [kMaxNodes] right-hand side of the sweeps
constexpr size_t kOffD0 = kOffB + 4ull * kMaxNodes;  // float  [kMaxNodes] sweep buffer
constexpr size_t kOffD1 = kOffD0 + 4ull * kMaxNodes; // float  [kMaxNodes] sweep buffer
constexpr size_t kOffPart = kOffD1 + 4ull * kMaxNodes; // double [kPartBlocks]
constexpr size_t kScratchBytes = kOffPart + 8ull * kPartBlocks;  // about 12 MiB

// Shared by every call on a device; holds the previous call's contents.
static __device__ __align__(256) unsigned char g_solve_scratch[kScratchBytes];

// Most kernel launches one call may issue (sweeps and residual passes).
constexpr long long kMaxLaunches = 1000000;

// Device address of the scratch array in the current device's context,
// looked up on every call: the lookup is cheap once the module is loaded, and
// a cached address would go stale if the context were reset or replaced
// between calls.  The first call in a context loads the module there.
cudaError_t scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

__global__ void k_na_init(int n, const float *__restrict__ s, double *__restrict__ x, float *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = 0.0;
    b[i] = s[i];
}

// y = b + K v, one warp per row, plain loads (any CSR layout)
__global__ void k_na_sweep(int n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                           const float *__restrict__ val, const float *__restrict__ b, const float *__restrict__ v,
                           float *__restrict__ y) {
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= n) return;
    float acc = 0.f;
    for (int e = row_ptr[row] + lane; e < row_ptr[row + 1]; e += 32) acc += val[e] * v[col[e]];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = b[row] + acc;
}

__global__ void k_na_update(int n, const float *__restrict__ d, double *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += (double)d[i];
}

// r = s - x + K x in FP64; b = (float) r; per-block sums of r^2 into part
__global__ void k_na_residual(int n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                              const float *__restrict__ val, const float *__restrict__ s,
                              const double *__restrict__ x, float *__restrict__ b, double *__restrict__ part) {
    __shared__ double red[8];
    const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double loc = 0.0;
    for (int row = blockIdx.x * warps + w; row < n; row += gridDim.x * warps) {
        double acc = 0.0;
        for (int e = row_ptr[row] + lane; e < row_ptr[row + 1]; e += 32) acc += (double)val[e] * x[col[e]];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            double r = (double)s[row] - x[row] + acc;
            b[row] = (float)r;
            loc += r * r;
        }
    }
    if (lane == 0) red[w] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < warps; ++i) t += red[i];
        part[blockIdx.x] = t;
    }
}

__global__ void k_na_final(const double *__restrict__ part, int nb, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += part[i];
    *out = t;
}

}  // namespace

extern "C" tursca_status tursca_csr_solve_noalloc(const int32_t *row_ptr, const int32_t *col, const float *val,
                                                  int n_nodes, const float *s, double *x, int sweeps,
                                                  int refinements, double *resid2, void *cuda_stream) {
    if (!row_ptr || !col || !val || !s || !x) return TURSCA_E_INVALID;
    if (n_nodes < 1 || n_nodes > kMaxNodes) return TURSCA_E_INVALID;
    if (sweeps < 0 || sweeps > 100000 || refinements < 1 || refinements > 1000) return TURSCA_E_INVALID;
    if ((long long)(sweeps + 2) * refinements + 2 > kMaxLaunches) return TURSCA_E_INVALID;
    // an error left pending by earlier work belongs to its owner: report it
    // without clearing it, before launching anything
    if (cudaPeekAtLastError() != cudaSuccess) return TURSCA_E_CUDA;
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return TURSCA_E_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char *p = (unsigned char *)base;
    float *b = (float *)(p + kOffB), *d0 = (float *)(p + kOffD0), *d1 = (float *)(p + kOffD1);
    double *part = (double *)(p + kOffPart);
    const int th = 256;
    const int nvec = (n_nodes + th - 1) / th;
    const long long rows_blocks = ((long long)n_nodes * 32 + th - 1) / th;
    int nres = (n_nodes + 7) / 8;
    if (nres > kPartBlocks) nres = kPartBlocks;
    k_na_init<<<nvec, th, 0, st>>>(n_nodes, s, x, b);
    // a launch that fails (a bad stream, say) fails them all: stop at the first
    if (cudaGetLastError() != cudaSuccess) return TURSCA_E_CUDA;
    for (int r = 0; r < refinements; ++r) {
        const float *cur = b;
        for (int k = 0; k < sweeps; ++k) {
            float *nxt = (k & 1) ? d1 : d0;
            k_na_sweep<<<(unsigned)rows_blocks, th, 0, st>>>(n_nodes, row_ptr, col, val, b, cur, nxt);
            cur = nxt;
        }
        k_na_update<<<nvec, th, 0, st>>>(n_nodes, cur, x);
        k_na_residual<<<nres, th, 0, st>>>(n_nodes, row_ptr, col, val, s, x, b, part);
    }
    if (resid2) k_na_final<<<1, 32, 0, st>>>(part, nres, resid2);
    return cudaGetLastError() == cudaSuccess ? TURSCA_OK : TURSCA_E_CUDA;
}
