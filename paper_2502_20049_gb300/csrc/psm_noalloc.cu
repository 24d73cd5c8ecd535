// psm_mass_noalloc: total mass of a caller-owned PDF field with no device
// allocation.  The library's other entry points allocate their scratch with
// cudaMalloc when a handle is created; this one keeps its scratch (per-block
// FP64 partial sums, a ticket counter and the result) in a file-scope
// __device__ array instead, for callers that must not allocate device memory
// (an application that routes every device allocation through its own pool,
// or a loop that cannot afford cudaMalloc's implicit device synchronisation).
#include <cmath>
#include <cstring>
#include <mutex>

#include "psm_kernels.cuh"

namespace psm {

constexpr int NOALLOC_CELLS_PER_BLOCK = 65536;  // fixed chunk: the summation order never changes
constexpr int NOALLOC_MAX_BLOCKS = 16384;       // 16384 * 65536 = 2^30 cells at most

// Layout: [0, NOALLOC_MAX_BLOCKS) block partials, [NOALLOC_MAX_BLOCKS] the
// result, [NOALLOC_MAX_BLOCKS + 1] holds the ticket counter (as an unsigned
// int).  Every GPU that loads the library holds this array (128 KB + 16 B)
// until the process exits.
constexpr int NOALLOC_SCRATCH_DOUBLES = NOALLOC_MAX_BLOCKS + 2;
static_assert(NOALLOC_SCRATCH_DOUBLES == NOALLOC_MAX_BLOCKS + 2, "partials, the result and the ticket");
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

struct NoAllocScratch {
  double* partials;
  double* result;
  unsigned int* ticket;
};

template <class S, int Q>
__global__ void __launch_bounds__(PSM_THREADS) k_mass_noalloc(const S* __restrict__ f, long long ncell, double rho0,
                                                              NoAllocScratch scr) {
  using T = typename Store<S>::T;
  const long long c0 = (long long)blockIdx.x * NOALLOC_CELLS_PER_BLOCK;
  long long c1 = c0 + NOALLOC_CELLS_PER_BLOCK;
  if (c1 > ncell) c1 = ncell;
  double acc = 0.0;
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    double m = rho0;
#pragma unroll
    for (int i = 0; i < Q; ++i) m += (double)Store<S>::ld(f + (long long)i * ncell + c);
    acc += m;
  }
  __shared__ double s_w[PSM_THREADS / 32];
  __shared__ double blk[1];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < PSM_THREADS / 32; ++w) s += s_w[w];
    blk[0] = s;
  }
  __syncthreads();
  grid_reduce(blk, 1, scr.partials, scr.ticket, scr.result);
}

namespace {

// Device address of g_noalloc_scratch, looked up once per device (in host code
// the symbol's name is only a stand-in for the device array).
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[64] = {};

cudaError_t scratch_for_current_device(NoAllocScratch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = ptr;
  }
  double* base = g_noalloc_ptr[dev];
  out->partials = base;
  out->result = base + NOALLOC_MAX_BLOCKS;
  out->ticket = reinterpret_cast<unsigned int*>(base + NOALLOC_MAX_BLOCKS + 1);
  return cudaSuccess;
}

template <class S>
cudaError_t launch_noalloc(int Q, const void* f, long long ncell, double rho0, NoAllocScratch scr, int blocks,
                           cudaStream_t st) {
  if (Q == 19)
    k_mass_noalloc<S, 19><<<blocks, PSM_THREADS, 0, st>>>(static_cast<const S*>(f), ncell, rho0, scr);
  else
    k_mass_noalloc<S, 27><<<blocks, PSM_THREADS, 0, st>>>(static_cast<const S*>(f), ncell, rho0, scr);
  return cudaGetLastError();
}

}  // namespace

int set_error(int code, const char* msg);

}  // namespace psm

extern "C" int psm_mass_noalloc(const void* f, int storage, int stencil, int64_t ncell, double rho0, void* stream,
                                double* out) {
  using namespace psm;
  if (!f || !out) return set_error(PSM_ERR_ARG, "psm_mass_noalloc: NULL argument");
  if (stencil != PSM_D3Q19 && stencil != PSM_D3Q27) return set_error(PSM_ERR_ARG, "stencil must be 19 or 27");
  if (storage < PSM_FP64 || storage > PSM_BF16_SHIFTED) return set_error(PSM_ERR_ARG, "bad storage");
  if (ncell < 1) return set_error(PSM_ERR_ARG, "psm_mass_noalloc: ncell must be >= 1");
  if (ncell > (int64_t)NOALLOC_MAX_BLOCKS * NOALLOC_CELLS_PER_BLOCK)
    return set_error(PSM_ERR_ARG,
                     "psm_mass_noalloc: ncell exceeds the static scratch limit of 2^30 cells "
                     "(16384 block partials of 65536 cells)");
  const int bytes = storage == PSM_FP64 ? 8 : (storage == PSM_FP32 ? 4 : 2);
  // f must be device memory of the current device holding Q * ncell values: a
  // host pointer would fault the kernel
  int rc = check_device_buffer(f, (size_t)stencil * (size_t)ncell * (size_t)bytes, "psm_mass_noalloc: f");
  if (rc != PSM_OK) return rc;
  NoAllocScratch scr;
  cudaError_t e = scratch_for_current_device(&scr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(PSM_ERR_CUDA, "psm_mass_noalloc: cannot resolve the static scratch address");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long blocks = (ncell + NOALLOC_CELLS_PER_BLOCK - 1) / NOALLOC_CELLS_PER_BLOCK;
  // one partial per block: the array holds NOALLOC_MAX_BLOCKS of them
  if (blocks > NOALLOC_MAX_BLOCKS) return set_error(PSM_ERR_ARG, "psm_mass_noalloc: too many blocks for the scratch");
  // the ticket must start at zero (the last block also resets it)
  e = cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) {
    switch (storage) {
      case PSM_FP64: e = launch_noalloc<double>(stencil, f, ncell, rho0, scr, (int)blocks, st); break;
      case PSM_FP32: e = launch_noalloc<float>(stencil, f, ncell, rho0, scr, (int)blocks, st); break;
      case PSM_FP16_SHIFTED: e = launch_noalloc<__half>(stencil, f, ncell, rho0, scr, (int)blocks, st); break;
      default: e = launch_noalloc<__nv_bfloat16>(stencil, f, ncell, rho0, scr, (int)blocks, st); break;
    }
  }
  // the result is read once, on `stream`, into a host local; it is tested
  // there and then written to out (a host store, or one more copy on `stream`
  // when out is device memory)
  double v = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, scr.result, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(PSM_ERR_CUDA, "psm_mass_noalloc: kernel or copy failed");
  }
  cudaPointerAttributes a;
  const bool out_dev = cudaPointerGetAttributes(&a, out) == cudaSuccess &&
                       (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (out_dev) {
    e = cudaMemcpyAsync(out, &v, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(PSM_ERR_CUDA, "psm_mass_noalloc: copy of the result failed");
    }
  } else {
    *out = v;
  }
  if (!std::isfinite(v)) return set_error(PSM_ERR_NONFINITE, "psm_mass_noalloc: the sum is NaN or Inf");
  return PSM_OK;
}
