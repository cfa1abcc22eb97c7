// noalloc.cu -- an energy entry point that performs no device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// solvation energy: an engine whose own allocator owns all device memory (and
// forbids cudaMalloc behind its back), or an MD driver that hands the library only
// the solution vector it already holds.  For them ddlpb_energy_noalloc computes the
// energy from caller buffers, using as scratch a fixed file-scope device array
// instead of memory of its own.  The call ends with a synchronisation of the
// caller's stream (the result is in *e on return), so it is not for use inside a
// stream capture or a host callback.
//
// The device address of the array is looked up once per device index and kept for
// the life of the process; this assumes the device's primary context (the one the
// runtime uses) is not reset in between (after cudaDeviceReset the cached address
// would be stale).
#include <mutex>

#include "common.cuh"

#define NA_BLOCK 256
#define NA_MAX_BLOCKS 4096   // scratch: one partial sum per block, plus the result
#define NA_MAX_ATOMS (NA_BLOCK * NA_MAX_BLOCKS)
#define NA_MAX_DEVICES 64

// Shared by every call on a device; holds the last call's partial sums and result
// until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS + 1];

// Pass 1: partial[b] = sum over the atoms of block b of q_j X_r[j, 00].
__global__ void k_na_partial(int n, int nb, const double* __restrict__ q, const double* __restrict__ X,
                             double* __restrict__ partial) {
    __shared__ double red[NA_BLOCK / 32];
    int j = blockIdx.x * NA_BLOCK + threadIdx.x;
    double s = j < n ? q[j] * X[(size_t)j * nb] : 0.0;
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < NA_BLOCK / 32; ++k) t += red[k];
        partial[blockIdx.x] = t;
    }
}

// Pass 2: result = 1/2 Y_00 sum_b partial[b].
__global__ void k_na_final(int blocks, double* __restrict__ scratch) {
    __shared__ double red[NA_BLOCK / 32];
    double s = 0;
    for (int b = threadIdx.x; b < blocks; b += NA_BLOCK) s += scratch[b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < NA_BLOCK / 32; ++k) t += red[k];
        scratch[NA_MAX_BLOCKS] = 0.5 * 0.28209479177387814 * t;
    }
}

static std::mutex g_na_mutex;
static double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

static thread_local std::string g_na_err;

extern "C" const char* ddlpb_noalloc_last_error(void) { return g_na_err.c_str(); }

extern "C" ddlpb_status ddlpb_energy_noalloc(int n, int lmax, const double* charges, const double* X, double* e,
                                             void* cuda_stream) {
    g_na_err.clear();
    if (!charges || !X || !e) {
        g_na_err = "NULL argument";
        return DDLPB_EINVAL;
    }
    if (n < 1 || n > NA_MAX_ATOMS) {
        g_na_err = "n must be in [1, " + std::to_string(NA_MAX_ATOMS) + "] (size of the static scratch)";
        return DDLPB_EINVAL;
    }
    if (lmax < 0 || lmax > DDLPB_LMAX_MAX) {
        g_na_err = "lmax out of range [0, 16]";
        return DDLPB_EINVAL;
    }
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) {
        g_na_err = std::string("cudaGetDevice: ") + cudaGetErrorString(err);
        return DDLPB_ECUDA;
    }
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        g_na_err = "device index " + std::to_string(dev) + " exceeds " + std::to_string(NA_MAX_DEVICES - 1);
        return DDLPB_EINVAL;
    }
    double* scratch = nullptr;
    {
        // Once per device, with that device current: the device address of the static
        // array (its host-side name is only a stand-in and must not reach a kernel).
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (err != cudaSuccess || !p) {
                g_na_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(err);
                return DDLPB_ECUDA;
            }
            g_na_ptr[dev] = (double*)p;
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nb = (lmax + 1) * (lmax + 1);
    const int blocks = (n + NA_BLOCK - 1) / NA_BLOCK;
    k_na_partial<<<blocks, NA_BLOCK, 0, st>>>(n, nb, charges, X, scratch);
    k_na_final<<<1, NA_BLOCK, 0, st>>>(blocks, scratch);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(e, scratch + NA_MAX_BLOCKS, sizeof(double), cudaMemcpyDefault, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) {
        g_na_err = std::string("CUDA: ") + cudaGetErrorString(err);
        return DDLPB_ECUDA;
    }
    return DDLPB_OK;
}
