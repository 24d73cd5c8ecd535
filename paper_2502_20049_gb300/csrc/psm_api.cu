// Host side of the libpsm C ABI (include/psm.h): handle, validation, device
// memory, per-step body poses (Sec. 3), kernel dispatch and the diagnostics.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "psm_adjoint.cuh"
#include "psm_kernels.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  return fail(e == cudaErrorMemoryAllocation ? PSM_ERR_OOM : PSM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PSM_CUDA(call, what)                      \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t storage_bytes(int st) {
  switch (st) {
    case PSM_FP64: return 8;
    case PSM_FP32: return 4;
    default: return 2;
  }
}

// Tensor maps of one PDF buffer (x, y, z, slot): boxes (TX, TY, 1, Q),
// (TX, 1, 1, 1) and (32, 1, 1, Q).
struct BufMaps {
  CUtensorMap tile;
  CUtensorMap row1;
  CUtensorMap warpq;
};

struct HostBody {
  unsigned long long* d_bricks = nullptr;
  unsigned char* d_occ = nullptr;  // occupancy (DevBody::occ)
  unsigned* d_occ8 = nullptr;      // block occupancy bits (DevBody::occ8)
  int64_t gx = 0, gy = 0, gz = 0;
  int s = 0, wpb = 1;
  double lo[3] = {0, 0, 0};
  double Q0[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double R0[3] = {0, 0, 0};
  double omega[3] = {0, 0, 0};
  double v[3] = {0, 0, 0};
  // angular velocity in u_s = omega x r + v (psm_set_us_omega); the pose
  // sequence keeps `omega`
  double us_omega[3] = {0, 0, 0};
};

// Pose at step n: Q_n = Rot(k, th) Q0 with k = omega/|omega|, th = |omega| n
// (Rodrigues: cos(th) I + sin(th) [k]x + (1 - cos(th)) k k^T), R_n = R0 + v n.
void body_pose(const HostBody& b, int64_t n, double Q[9], double R[3]) {
  const double wn = std::sqrt(b.omega[0] * b.omega[0] + b.omega[1] * b.omega[1] + b.omega[2] * b.omega[2]);
  double Rt[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (wn > 0.0) {
    const double k0 = b.omega[0] / wn, k1 = b.omega[1] / wn, k2 = b.omega[2] / wn;
    const double th = wn * double(n);
    const double c = std::cos(th), s = std::sin(th), oc = 1.0 - c;
    Rt[0] = c + oc * k0 * k0;
    Rt[1] = oc * k0 * k1 - s * k2;
    Rt[2] = oc * k0 * k2 + s * k1;
    Rt[3] = oc * k1 * k0 + s * k2;
    Rt[4] = c + oc * k1 * k1;
    Rt[5] = oc * k1 * k2 - s * k0;
    Rt[6] = oc * k2 * k0 - s * k1;
    Rt[7] = oc * k2 * k1 + s * k0;
    Rt[8] = c + oc * k2 * k2;
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      Q[3 * r + c] = (Rt[3 * r + 0] * b.Q0[0 + c] + Rt[3 * r + 1] * b.Q0[3 + c]) + Rt[3 * r + 2] * b.Q0[6 + c];
  for (int k = 0; k < 3; ++k) R[k] = b.R0[k] + b.v[k] * double(n);
}

}  // namespace

struct psm_solver {
  psm_grid grid;
  psm_lattice lat;
  psm_collision col;
  psm::Grid3 g;
  psm::Tiling tiling;
  cudaStream_t stream = nullptr;
  int Q = 19;
  void* buf[2] = {nullptr, nullptr};
  bool owns_buf = true;  // false: caller-owned PDF buffers (psm_create_with_buffers)
  int cur = 0;
  int64_t step = 0;
  int nbodies = 0;
  HostBody body[PSM_MAX_BODIES];
  // psm_set_remap(h, 0): every later step uses the body poses of step frozen_step
  bool remap_frozen = false;
  int64_t frozen_step = 0;
  // two-way coupled bodies (bit b): their state and next-step DevBody on the device
  unsigned free_mask = 0;
  psm::BodyDyn* d_dyn = nullptr;
  psm::DevBody* d_dev_bodies = nullptr;
  double ghost[27];
  int max_blocks = 0;
  double* d_partials = nullptr;
  unsigned int* d_ticket = nullptr;
  double* d_series = nullptr;
  int64_t cap = 0;
  double* d_sum = nullptr;
  float* d_delta = nullptr;
  int* d_err = nullptr;
  // TMA-staged step kernel: eligibility, its tiling and the tensor maps per buffer
  bool tma_ok = false;
  bool tma_odd_ok = false;  // the AA odd step has its TMA variant too (full 256-cell rows)
  int variant = PSM_KERNEL_AUTO;
  psm::Tiling tma_tiling;      // the solver's two-grid or AA even steps
  psm::Tiling tma_tiling_odd;  // AA odd steps (one cell per thread)
  psm::Tiling tma_tiling_tg;   // two-grid steps of the backward recompute
  bool tma_tg_ok = false;      // the backward recompute has its TMA variant
  BufMaps maps[2];
  // trajectory recording for psm_backward: checkpoints every rec_K steps from rec_n0
  bool recording = false;
  // psm_set_z_offset was called: the lattice is a z-slab of a larger domain
  bool slab = false;
  int rec_K = 0;
  int rec_flags = 0;
  int64_t rec_n0 = 0;
  std::vector<void*> ckpt;
  // recompute buffers of psm_backward (slot 0 unused: the checkpoint), kept
  // between calls, and their tensor maps
  std::vector<void*> rec_slots;
  std::vector<BufMaps> rec_maps;
  // a second set of recompute buffers and its stream: psm_backward recomputes
  // the segment before the current one while the adjoint sweeps the current
  // one (allocated when the device has room; otherwise one set, in sequence);
  // the recompute's force/torque sums go to their own grid-reduction scratch
  std::vector<void*> rec_slots2;
  std::vector<BufMaps> rec_maps2;
  cudaStream_t rec_stream = nullptr;
  double* d_partials2 = nullptr;
  unsigned int* d_ticket2 = nullptr;
  void* rec_lam[2] = {nullptr, nullptr};  // the two adjoint fields
  double* rec_grad = nullptr;             // dJ/d delta accumulator
};

namespace psm {

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

namespace {
using MemRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
// cuMemGetAddressRange through the runtime's driver entry points (nullptr if
// the driver does not provide it)
MemRangeFn mem_range_fn() {
  static MemRangeFn fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &ptr, 3020, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      ptr = nullptr;
    }
    return reinterpret_cast<MemRangeFn>(ptr);
  }();
  return fn;
}
}  // namespace

int check_device_buffer(const void* p, size_t bytes, const char* what) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PSM_ERR_ARG, "%s: cannot tell whether it is device memory (%s)", what, cudaGetErrorString(e));
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(PSM_ERR_ARG, "%s: not device memory (%s)", what,
                a.type == cudaMemoryTypeHost ? "page-locked host memory" : "host memory");
  int dev = -1;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PSM_ERR_ARG, "%s: no current device (%s)", what, cudaGetErrorString(e));
  }
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    return fail(PSM_ERR_ARG, "%s: memory of device %d, the current device is %d", what, a.device, dev);
  if (MemRangeFn fn = mem_range_fn()) {
    CUdeviceptr base = 0;
    size_t size = 0;
    if (fn(&base, &size, (CUdeviceptr)(uintptr_t)p) == CUDA_SUCCESS) {
      const unsigned long long q = (unsigned long long)(uintptr_t)p, b0 = (unsigned long long)base;
      if (q < b0 || q - b0 > size || size - (q - b0) < bytes)
        return fail(PSM_ERR_ARG, "%s: %llu bytes needed, its allocation holds %llu bytes from this address", what,
                    (unsigned long long)bytes, (unsigned long long)(q >= b0 && q - b0 <= size ? size - (q - b0) : 0));
    } else {
      cudaGetLastError();
    }
  }
  return PSM_OK;
}

void set_slots(StepParams& p, int storage, int Q) {
  const size_t b = storage == PSM_FP64 ? 8 : (storage == PSM_FP32 ? 4 : 2);
  char* src = static_cast<char*>(p.f);
  char* dst = static_cast<char*>(p.f_dst ? p.f_dst : p.f);
  for (int i = 0; i < 27; ++i) {
    p.src_slot[i] = i < Q ? src + (size_t)i * (size_t)p.g.ncell * b : nullptr;
    p.dst_slot[i] = i < Q ? dst + (size_t)i * (size_t)p.g.ncell * b : nullptr;
  }
}

// Tiles of tx x ty = PSM_THREADS cells (one per thread): tx is the smallest
// power of two >= nx from 32 up to PSM_THREADS, so that ty = PSM_THREADS / tx
// leaves no thread without a cell of its own tile (a tx that does not divide
// the block, such as 96, would give the spare threads cells of the next tile).
Tiling make_tiling(int nx, int ny, int nz) {
  Tiling t;
  int tx = 32;
  while (tx < nx && tx < PSM_THREADS) tx *= 2;
  t.tx = tx;
  t.ty = PSM_THREADS / tx;
  t.ntx = (nx + t.tx - 1) / t.tx;
  t.nty = (ny + t.ty - 1) / t.ty;
  t.ntiles = (long long)t.ntx * t.nty * nz;
  return t;
}

cudaError_t launch_step(int storage, int Q, int mode, const StepParams& p, cudaStream_t st) {
  switch (storage) {
    case PSM_FP64: return launch_step_fp64(Q, mode, p.fluid, p, st);
    case PSM_FP32: return launch_step_fp32(Q, mode, p.fluid, p, st);
    case PSM_FP16_SHIFTED: return launch_step_fp16(Q, mode, p.fluid, p, st);
    default: return launch_step_bf16(Q, mode, p.fluid, p, st);
  }
}
cudaError_t launch_step_tma(int storage, int Q, int mode, const StepParams& p, const TmaMaps& m, cudaStream_t st) {
  switch (storage) {
    case PSM_FP64: return launch_step_tma_fp64(Q, mode, p.fluid, p, m, st);
    case PSM_FP32: return launch_step_tma_fp32(Q, mode, p.fluid, p, m, st);
    case PSM_FP16_SHIFTED: return launch_step_tma_fp16(Q, mode, p.fluid, p, m, st);
    default: return launch_step_tma_bf16(Q, mode, p.fluid, p, m, st);
  }
}
int tma_smem_bytes(int storage, int Q, int mode, int fl) {
  switch (storage) {
    case PSM_FP64: return tma_smem_bytes_fp64(Q, mode, fl);
    case PSM_FP32: return tma_smem_bytes_fp32(Q, mode, fl);
    case PSM_FP16_SHIFTED: return tma_smem_bytes_fp16(Q, mode, fl);
    default: return tma_smem_bytes_bf16(Q, mode, fl);
  }
}
#define PSM_IO_DISPATCH(FN)                                                    \
  cudaError_t launch_##FN(int storage, int Q, const IoParams& p, cudaStream_t st) { \
    switch (storage) {                                                         \
      case PSM_FP64: return launch_##FN##_fp64(Q, p, st);                      \
      case PSM_FP32: return launch_##FN##_fp32(Q, p, st);                      \
      case PSM_FP16_SHIFTED: return launch_##FN##_fp16(Q, p, st);              \
      default: return launch_##FN##_bf16(Q, p, st);                            \
    }                                                                          \
  }
PSM_IO_DISPATCH(import)
PSM_IO_DISPATCH(export)
PSM_IO_DISPATCH(export_raw)
PSM_IO_DISPATCH(macro)
cudaError_t launch_mass(int storage, int Q, const IoParams& p, int blocks, cudaStream_t st) {
  switch (storage) {
    case PSM_FP64: return launch_mass_fp64(Q, p, blocks, st);
    case PSM_FP32: return launch_mass_fp32(Q, p, blocks, st);
    case PSM_FP16_SHIFTED: return launch_mass_fp16(Q, p, blocks, st);
    default: return launch_mass_bf16(Q, p, blocks, st);
  }
}

__global__ void k_remap(const __grid_constant__ RemapParams p) {
  const long long plane = (long long)p.g.nx * p.g.ny;
  const long long n = plane * (p.z_end - p.z_begin);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int z = p.z_begin + (int)(idx / plane);
    const long long r = idx % plane;
    const int y = (int)(r / p.g.nx), x = (int)(r % p.g.nx);
    int owner;
    p.eps_out[idx] = cell_eps(p.body, p.nbodies, x, y, z + p.g.z0, owner);
  }
}

// every element of dst[0, n) = v in the storage type (psm_fill_slot_plane)
template <class S>
__global__ void k_fill_plane(S* dst, long long n, double v) {
  const S sv = Store<S>::from_double(v);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = sv;
}

// one thread per occupancy cell c in [-1, g - 1]^3
__global__ void k_occupancy(const unsigned long long* __restrict__ bricks, int gx, int gy, int gz, int wpb,
                            unsigned char* __restrict__ occ) {
  const long long n = (long long)(gx + 1) * (gy + 1) * (gz + 1);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int cx = (int)(idx % (gx + 1)) - 1;
    const int cy = (int)((idx / (gx + 1)) % (gy + 1)) - 1;
    const int cz = (int)(idx / ((long long)(gx + 1) * (gy + 1))) - 1;
    unsigned long long any = 0ull;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int x = cx + dx, y = cy + dy, z = cz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= gx || y >= gy || z >= gz) continue;
          const unsigned long long* w = bricks + (((long long)z * gy + y) * gx + x) * wpb;
          for (int k = 0; k < wpb; ++k) any |= w[k];
        }
    occ[idx] = any ? 1 : 0;
  }
}

// one thread per block of 8^3 occupancy bytes: its bit is set iff a byte is
__global__ void k_occupancy8(const unsigned char* __restrict__ occ, int ox, int oy, int oz, unsigned* occ8) {
  const int bx = (ox + 7) / 8, by = (oy + 7) / 8, bz = (oz + 7) / 8;
  const long long n = (long long)bx * by * bz;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % bx), iy = (int)((idx / bx) % by), iz = (int)(idx / ((long long)bx * by));
    bool any = false;
    for (int z = iz * 8; z < iz * 8 + 8 && z < oz && !any; ++z)
      for (int y = iy * 8; y < iy * 8 + 8 && y < oy && !any; ++y)
        for (int x = ix * 8; x < ix * 8 + 8 && x < ox; ++x)
          if (occ[((long long)z * oy + y) * ox + x]) {
            any = true;
            break;
          }
    if (any) atomicOr(occ8 + (idx >> 5), 1u << (idx & 31));
  }
}

cudaError_t launch_occupancy8(const unsigned char* occ, int ox, int oy, int oz, unsigned* occ8, cudaStream_t st) {
  const long long n = (long long)((ox + 7) / 8) * ((oy + 7) / 8) * ((oz + 7) / 8);
  long long b = (n + PSM_THREADS - 1) / PSM_THREADS;
  if (b > 4096) b = 4096;
  k_occupancy8<<<(int)(b < 1 ? 1 : b), PSM_THREADS, 0, st>>>(occ, ox, oy, oz, occ8);
  return cudaGetLastError();
}

cudaError_t launch_occupancy(const unsigned long long* bricks, int gx, int gy, int gz, int wpb, unsigned char* occ,
                             cudaStream_t st) {
  const long long n = (long long)(gx + 1) * (gy + 1) * (gz + 1);
  long long b = (n + PSM_THREADS - 1) / PSM_THREADS;
  if (b > 4096) b = 4096;
  k_occupancy<<<(int)(b < 1 ? 1 : b), PSM_THREADS, 0, st>>>(bricks, gx, gy, gz, wpb, occ);
  return cudaGetLastError();
}

// One semi-implicit Euler step of the rigid-body equations per body in mask
// (thread b), from this step's force and torque on the body ft[b][6]:
//   v += (F + Fext) / m,  R += v,  L += T + Text,
//   Q <- Rot(w*) Q, w* = Q Ib^-1 Q^T L,  w = Q Ib^-1 Q^T L,
// then the DevBody of the next step (kinematics, the cell box of the rotated
// geometry box widened by 2.5 cells, the remap's pose and its float form).
__device__ void q_ibinv_qt(const double* Q, const double* Ibinv, const double* L, double* w) {
  double a[3], b[3];
  for (int i = 0; i < 3; ++i) a[i] = Q[i] * L[0] + Q[3 + i] * L[1] + Q[6 + i] * L[2];
  for (int i = 0; i < 3; ++i) b[i] = Ibinv[3 * i] * a[0] + Ibinv[3 * i + 1] * a[1] + Ibinv[3 * i + 2] * a[2];
  for (int i = 0; i < 3; ++i) w[i] = Q[3 * i] * b[0] + Q[3 * i + 1] * b[1] + Q[3 * i + 2] * b[2];
}

__global__ void k_body_update(BodyDyn* dyn, DevBody* dev, const double* ft, unsigned mask, int nb, int nx, int ny,
                              int nz) {
  const int b = threadIdx.x;
  if (b >= nb || !((mask >> b) & 1u)) return;
  BodyDyn& S = dyn[b];
  const double* F = ft + 6 * b;
  for (int k = 0; k < 3; ++k) S.v[k] += (F[k] + S.Fext[k]) / S.mass;
  for (int k = 0; k < 3; ++k) S.R[k] += S.v[k];
  for (int k = 0; k < 3; ++k) S.L[k] += F[3 + k] + S.Text[k];
  double ws[3];
  q_ibinv_qt(S.Q, S.Ibinv, S.L, ws);
  const double a = sqrt(ws[0] * ws[0] + ws[1] * ws[1] + ws[2] * ws[2]);
  if (a > 0.0) {
    const double k0 = ws[0] / a, k1 = ws[1] / a, k2 = ws[2] / a;
    double sn, cs;
    sincos(a, &sn, &cs);
    const double oc = 1.0 - cs;
    const double Rm[9] = {cs + oc * k0 * k0,      oc * k0 * k1 - sn * k2, oc * k0 * k2 + sn * k1,
                          oc * k1 * k0 + sn * k2, cs + oc * k1 * k1,      oc * k1 * k2 - sn * k0,
                          oc * k2 * k0 - sn * k1, oc * k2 * k1 + sn * k0, cs + oc * k2 * k2};
    double Qn[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Qn[3 * r + c] = Rm[3 * r] * S.Q[c] + Rm[3 * r + 1] * S.Q[3 + c] + Rm[3 * r + 2] * S.Q[6 + c];
    for (int k = 0; k < 9; ++k) S.Q[k] = Qn[k];
  }
  q_ibinv_qt(S.Q, S.Ibinv, S.L, S.w);
  DevBody& d = dev[b];
  for (int k = 0; k < 3; ++k) {
    d.Rf[k] = (float)S.R[k];
    d.R[k] = S.R[k];
    d.omega[k] = S.w[k];
    d.v[k] = S.v[k];
    d.omegaf[k] = (float)S.w[k];
    d.vf[k] = (float)S.v[k];
  }
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  const double ext[3] = {(double)S.gx, (double)S.gy, (double)S.gz};
  for (int c = 0; c < 8; ++c) {
    double pb[3];
    for (int k = 0; k < 3; ++k) pb[k] = S.lo[k] + (((c >> k) & 1) ? ext[k] : 0.0);
    for (int r = 0; r < 3; ++r) {
      const double w = S.Q[3 * r] * pb[0] + S.Q[3 * r + 1] * pb[1] + S.Q[3 * r + 2] * pb[2] + S.R[r];
      mn[r] = fmin(mn[r], w);
      mx[r] = fmax(mx[r], w);
    }
  }
  const int dims[3] = {nx, ny, nz};
  int lo_[3], hi_[3];
  for (int k = 0; k < 3; ++k) {
    double a0 = floor(mn[k] - 2.5), e = ceil(mx[k] + 2.5) + 1.0;
    if (a0 < 0) a0 = 0;
    if (e > (double)dims[k]) e = (double)dims[k];
    if (e < a0) e = a0;
    lo_[k] = (int)a0;
    hi_[k] = (int)e;
  }
  d.x0 = lo_[0];
  d.x1 = hi_[0];
  d.y0 = lo_[1];
  d.y1 = hi_[1];
  d.z0 = lo_[2];
  d.z1 = hi_[2];
  remap_setup(d, S.Q, S.R, S.lo);
}

cudaError_t launch_body_update(BodyDyn* dyn, DevBody* dev, const double* ft, unsigned mask, int nb, int nx, int ny,
                               int nz, cudaStream_t st) {
  k_body_update<<<1, 32, 0, st>>>(dyn, dev, ft, mask, nb, nx, ny, nz);
  return cudaGetLastError();
}

cudaError_t launch_remap(const RemapParams& p, cudaStream_t st) {
  long long cells = (long long)p.g.nx * p.g.ny * (p.z_end - p.z_begin);
  long long b = (cells + PSM_THREADS - 1) / PSM_THREADS;
  if (b > 4096) b = 4096;
  k_remap<<<(int)(b < 1 ? 1 : b), PSM_THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace psm

namespace {

using psm::DevBody;
using psm::IoParams;
using psm::StepParams;

void fill_ghost(psm_solver* h) {
  const double* u = h->grid.u_in;
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < 27; ++i) h->ghost[i] = 0.0;
  for (int i = 0; i < h->Q; ++i) {
    const double w = h->Q == 19 ? psm::lat_w<19>(i) : psm::lat_w<27>(i);
    const double cu = psm::lat_cx(i) * u[0] + psm::lat_cy(i) * u[1] + psm::lat_cz(i) * u[2];
    const double fe = w * h->grid.rho0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    h->ghost[i] = fe - w * h->grid.rho0;
  }
}

// Device view of body b at step n, including the world box of cells whose
// eps can be non-zero: the axis-aligned hull of the rotated geometry box,
// widened by 2.5 cells (a cell's sub-cell block reaches at most
// sqrt(3) (1/2 + 2^-s / 2) < 1.75 from its centre).
DevBody dev_body(const psm_solver* h, int bi, int64_t n) {
  const HostBody& b = h->body[bi];
  DevBody d;
  std::memset(&d, 0, sizeof d);
  double Q[9], R[3];
  body_pose(b, h->remap_frozen ? h->frozen_step : n, Q, R);
  d.bricks = b.d_bricks;
  d.occ = b.d_occ;
  d.occ8 = b.d_occ8;
  d.o8x = (int)((b.gx + 1 + 7) / 8);
  d.o8y = (int)((b.gy + 1 + 7) / 8);
  d.gx = (int)b.gx;
  d.gy = (int)b.gy;
  d.gz = (int)b.gz;
  d.s = b.s;
  d.wpb = b.wpb;
  for (int k = 0; k < 3; ++k) {
    d.Rf[k] = (float)R[k];
    d.R[k] = R[k];
    d.omega[k] = b.us_omega[k];
    d.v[k] = b.v[k];
    d.omegaf[k] = (float)b.us_omega[k];
    d.vf[k] = (float)b.v[k];
  }
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  const double ext[3] = {(double)b.gx, (double)b.gy, (double)b.gz};
  for (int c = 0; c < 8; ++c) {
    double pb[3];
    for (int k = 0; k < 3; ++k) pb[k] = b.lo[k] + (((c >> k) & 1) ? ext[k] : 0.0);
    for (int r = 0; r < 3; ++r) {
      const double w = Q[3 * r + 0] * pb[0] + Q[3 * r + 1] * pb[1] + Q[3 * r + 2] * pb[2] + R[r];
      mn[r] = std::fmin(mn[r], w);
      mx[r] = std::fmax(mx[r], w);
    }
  }
  // world cells of this grid: [0, nx) x [0, ny) x [z0, z0 + nz)
  const int64_t first[3] = {0, 0, h->g.z0};
  const int64_t dims[3] = {h->grid.nx, h->grid.ny, h->g.z0 + h->grid.nz};
  int lo_[3], hi_[3];
  for (int k = 0; k < 3; ++k) {
    double a = std::floor(mn[k] - 2.5), e = std::ceil(mx[k] + 2.5) + 1.0;
    if (a < (double)first[k]) a = (double)first[k];
    if (e > (double)dims[k]) e = (double)dims[k];
    if (e < a) e = a;
    lo_[k] = (int)a;
    hi_[k] = (int)e;
  }
  d.x0 = lo_[0];
  d.x1 = hi_[0];
  d.y0 = lo_[1];
  d.y1 = hi_[1];
  d.z0 = lo_[2];
  d.z1 = hi_[2];
  psm::remap_setup(d, Q, R, b.lo);
  return d;
}

// slot `slot` of plane z in the buffer the next step reads
void* slot_plane_addr(const psm_solver* h, int slot, int z) {
  void* buf = h->lat.streaming == PSM_STREAM_TWO_GRID ? h->buf[h->cur] : h->buf[0];
  const size_t plane = (size_t)h->grid.nx * (size_t)h->grid.ny;
  return static_cast<char*>(buf) + ((size_t)slot * (size_t)h->g.ncell + (size_t)z * plane) *
                                       storage_bytes(h->lat.storage);
}

int layout_of(const psm_solver* h) {
  if (h->lat.streaming == PSM_STREAM_TWO_GRID) return psm::LAYOUT_NATURAL;
  return (h->step & 1) ? psm::LAYOUT_SWAPPED : psm::LAYOUT_NATURAL;
}

void io_base(const psm_solver* h, IoParams& p) {
  std::memset(&p, 0, sizeof p);
  p.g = h->g;
  p.t = h->tiling;
  p.f = h->buf[h->cur];
  p.layout = layout_of(h);
  for (int i = 0; i < 27; ++i) p.ghost[i] = h->ghost[i];
  p.rho0 = h->grid.rho0;
}

// planes per chunk so that one chunk of `per_cell` bytes stays near 64 MiB
int chunk_planes(const psm_solver* h, size_t per_cell) {
  const size_t plane = (size_t)h->grid.nx * h->grid.ny * per_cell;
  size_t p = (64u << 20) / (plane ? plane : 1);
  if (p < 1) p = 1;
  if (p > (size_t)h->grid.nz) p = (size_t)h->grid.nz;
  return (int)p;
}

int import_uniform(psm_solver* h, double rho, const double u[3]) {
  IoParams p;
  io_base(h, p);
  p.uniform = 1;
  p.rho = rho;
  for (int k = 0; k < 3; ++k) p.u[k] = u[k];
  p.z_begin = 0;
  p.z_end = (int)h->grid.nz;
  PSM_CUDA(psm::launch_import(h->lat.storage, h->Q, p, h->stream), "import kernel");
  return PSM_OK;
}

bool valid_handle(psm_handle h) { return h != nullptr; }

// 1: under PSM_KERNEL_AUTO the AA odd step (per-direction rows) uses plain
// global loads even where its TMA-staged variant applies (0: the TMA variant,
// measured faster on GB300).
#ifndef PSM_AA_ODD_PLAIN
#define PSM_AA_ODD_PLAIN 0
#endif

// TMA shape rules (see k_step_tma): TX = min(256, nx), nx % TX == 0,
// 256 % nx == 0 if nx < 256, TY = 256 / TX divides ny, rows of 16-byte
// multiples, at least 32 cells per row segment, and the staging buffers of
// the modes used fit the shared memory a block may have.
// Tiling of the TMA step kernel in `mode`: tiles of TX = min(nx, 256) cells
// of TY rows, TX TY = 256 times the kernel's cells per thread.  false where
// the shape does not allow it.
bool tma_tiling_for(const psm_solver* h, int mode, psm::Tiling& t) {
  const int64_t nx = h->grid.nx, ny = h->grid.ny, nz = h->grid.nz;
  const int64_t b = (int64_t)storage_bytes(h->lat.storage);
  const int64_t TX = nx >= 256 ? 256 : nx;
  if (TX < 32 || nx % TX != 0 || (nx < 256 && 256 % nx != 0)) return false;
  const int64_t TY = (256 / TX) * psm::tma_cells_per_thread((int)b, mode, h->Q, h->col.fluid);
  if (ny % TY != 0 || (TX * b) % 16 != 0 || (nx * b) % 16 != 0) return false;
  t.tx = (int)TX;
  t.ty = (int)TY;
  t.ntx = (int)(nx / TX);
  t.nty = (int)(ny / TY);
  t.ntiles = (long long)t.ntx * t.nty * nz;
  return true;
}

bool tma_shape(const psm_solver* h, psm::Tiling& t, psm::Tiling& t_odd) {
  const int own_mode = h->lat.streaming == PSM_STREAM_TWO_GRID ? psm::MODE_TG : psm::MODE_AA_EVEN;
  if (!tma_tiling_for(h, own_mode, t)) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const int mode = h->lat.streaming == PSM_STREAM_TWO_GRID ? psm::MODE_TG : psm::MODE_AA_EVEN;
  if (psm::tma_smem_bytes(h->lat.storage, h->Q, mode, h->col.fluid) > optin) return false;
  if (!tma_tiling_for(h, psm::MODE_AA_ODD, t_odd)) return false;
  return true;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      ptr = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }();
  return fn;
}

// Tensor maps of PDF buffer `buf` as a (x, y, z, slot) tensor.
bool encode_maps(const psm_solver* h, void* buf, BufMaps& m, const psm::Tiling& tiling) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  CUtensorMapDataType dt = h->lat.storage == PSM_FP64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : h->lat.storage == PSM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : h->lat.storage == PSM_FP16_SHIFTED ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t b = storage_bytes(h->lat.storage);
  const cuuint64_t dims[4] = {(cuuint64_t)h->grid.nx, (cuuint64_t)h->grid.ny, (cuuint64_t)h->grid.nz,
                              (cuuint64_t)h->Q};
  const cuuint64_t strides[3] = {dims[0] * b, dims[0] * dims[1] * b, dims[0] * dims[1] * dims[2] * b};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  const cuuint32_t box_q[4] = {(cuuint32_t)tiling.tx, (cuuint32_t)tiling.ty, 1, (cuuint32_t)h->Q};
  const cuuint32_t box_1[4] = {(cuuint32_t)tiling.tx, 1, 1, 1};
  CUresult r1 = enc(&m.tile, dt, 4, buf, dims, strides, box_q, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = enc(&m.row1, dt, 4, buf, dims, strides, box_1, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  const cuuint32_t box_w[4] = {32, 1, 1, (cuuint32_t)h->Q};
  CUresult r3 = enc(&m.warpq, dt, 4, buf, dims, strides, box_w, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS && r3 == CUDA_SUCCESS;
}

template <class T>
void fill_consts(const psm_solver* h, psm::ConstT<T>& c) {
  c.rho0 = (T)h->grid.rho0;
  if (h->col.fluid == PSM_TRT) {
    const double wp = 1.0 / h->col.tau;
    const double wm = 1.0 / (h->col.trt_lambda / (h->col.tau - 0.5) + 0.5);
    c.om_a = (T)(0.5 * (wp + wm));
    c.om_b = (T)(0.5 * (wp - wm));
  } else {
    c.om_a = (T)(1.0 / h->col.tau);
    c.om_b = (T)0;
  }
  c.inv_tau = (T)(1.0 / h->col.tau);
  c.tmh = (T)(h->col.tau - 0.5);
  for (int i = 0; i < 27; ++i) c.ghost[i] = (T)h->ghost[i];
  double omp, omm;
  if (h->col.fluid == PSM_TRT) {
    omp = 1.0 / h->col.tau;
    omm = 1.0 / (h->col.trt_lambda / (h->col.tau - 0.5) + 0.5);
  } else {
    omp = omm = 1.0 / h->col.tau;
  }
  c.omp1 = (T)(1.0 - omp);
  c.hp1 = (T)(0.5 * (1.0 - omp));
  c.hm1 = (T)(0.5 * (1.0 - omm));
  // cumulant: 1 - rate for the shear, bulk, third- and fourth-order families
  c.cum1[0] = (T)(1.0 - 1.0 / h->col.tau);
  c.cum_unit = 1;
  for (int k = 0; k < 3; ++k) {
    const double w = h->col.cum_omega[k] == 0.0 ? 1.0 : h->col.cum_omega[k];
    c.cum1[k + 1] = (T)(1.0 - w);
    if (w != 1.0) c.cum_unit = 0;
  }
  // weight per class |c|^2 = 0..3 (D3Q19 has no corner directions)
  const double w19[4] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0, 0.0};
  const double w27[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
  for (int k = 0; k < 4; ++k) {
    const double w = h->Q == 19 ? w19[k] : w27[k];
    c.pw[k] = (T)(omp * w);
    c.pk[k] = (T)(4.5 * omp * w);
    c.pd[k] = (T)(3.0 * omm * w);
  }
}

// A kernel gave up on a bounded wait: report it once.
int check_err(psm_solver* h) {
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "error-flag read");
  if (flag) {
    cudaMemset(h->d_err, 0, sizeof(int));
    if (flag == 2) return fail(PSM_ERR_CUDA, "a step kernel was launched with a tiling it was not built for (results invalid)");
    return fail(PSM_ERR_CUDA, "a step kernel timed out waiting for its staged loads (results invalid)");
  }
  return PSM_OK;
}

size_t state_bytes(const psm_solver* h) {
  return (size_t)h->Q * (size_t)h->g.ncell * storage_bytes(h->lat.storage);
}

// copy the current natural-layout state into a new checkpoint (stream ordered)
int take_checkpoint(psm_solver* h) {
  void* c = nullptr;
  PSM_CUDA(cudaMallocAsync(&c, state_bytes(h), h->stream), "checkpoint allocation");
  const void* src = h->lat.streaming == PSM_STREAM_TWO_GRID ? h->buf[h->cur] : h->buf[0];
  cudaError_t e = cudaMemcpyAsync(c, src, state_bytes(h), cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(c, h->stream);
    return cuda_fail(e, "checkpoint copy");
  }
  h->ckpt.push_back(c);
  return PSM_OK;
}

void drop_checkpoints(psm_solver* h) {
  for (void* c : h->ckpt) cudaFreeAsync(c, h->stream);
  h->ckpt.clear();
}

cudaError_t launch_adjoint(int storage, int Q, int trt, const psm::AdjParams& p, cudaStream_t st) {
  switch (storage) {
    case PSM_FP64: return psm::launch_adjoint_fp64(Q, trt, p, st);
    case PSM_FP32: return psm::launch_adjoint_fp32(Q, trt, p, st);
    case PSM_FP16_SHIFTED: return psm::launch_adjoint_fp16(Q, trt, p, st);
    default: return psm::launch_adjoint_bf16(Q, trt, p, st);
  }
}
cudaError_t launch_adjoint_init(int storage, int Q, const psm::AdjParams& p, int blocks, cudaStream_t st) {
  switch (storage) {
    case PSM_FP64: return psm::launch_adjoint_init_fp64(Q, p, blocks, st);
    case PSM_FP32: return psm::launch_adjoint_init_fp32(Q, p, blocks, st);
    case PSM_FP16_SHIFTED: return psm::launch_adjoint_init_fp16(Q, p, blocks, st);
    default: return psm::launch_adjoint_init_bf16(Q, p, blocks, st);
  }
}

}  // namespace

extern "C" {

const char* psm_last_error(void) { return g_err.c_str(); }

int psm_lattice_velocities(int stencil, int* c_out, double* w_out, int* opp_out) {
  if (stencil != PSM_D3Q19 && stencil != PSM_D3Q27) return fail(PSM_ERR_ARG, "stencil must be 19 or 27");
  for (int i = 0; i < stencil; ++i) {
    if (c_out) {
      c_out[3 * i + 0] = psm::lat_cx(i);
      c_out[3 * i + 1] = psm::lat_cy(i);
      c_out[3 * i + 2] = psm::lat_cz(i);
    }
    if (w_out) w_out[i] = stencil == 19 ? psm::lat_w<19>(i) : psm::lat_w<27>(i);
    if (opp_out) opp_out[i] = psm::lat_opp(i);
  }
  return PSM_OK;
}

namespace {
// psm_create and psm_create_with_buffers: user_bufs (nullptr: allocate) hold
// the caller's PDF buffers; keep: their contents are the initial state.
int create_impl(const psm_grid* grid, const psm_lattice* lattice, const psm_collision* collision, void* stream,
                void* const* user_bufs, bool keep, psm_handle* out) {
  if (!grid || !lattice || !collision || !out) return fail(PSM_ERR_ARG, "psm_create: NULL argument");
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(PSM_ERR_ARG, "grid sizes must be >= 1");
  if (grid->nx > (1 << 30) || grid->ny > (1 << 30) || grid->nz > (1 << 30))
    return fail(PSM_ERR_ARG, "grid size per axis must be < 2^30");
  const double ncell = (double)grid->nx * (double)grid->ny * (double)grid->nz;
  if (ncell >= 4294967296.0) return fail(PSM_ERR_ARG, "nx*ny*nz must be < 2^32");
  if (grid->bc_z != PSM_BC_PERIODIC && grid->bc_z != PSM_BC_EQ_INLET_OUTLET) return fail(PSM_ERR_ARG, "bad bc_z");
  if (!(grid->rho0 > 0.0) || !std::isfinite(grid->rho0)) return fail(PSM_ERR_ARG, "rho0 must be > 0");
  const double un = std::sqrt(grid->u_in[0] * grid->u_in[0] + grid->u_in[1] * grid->u_in[1] +
                              grid->u_in[2] * grid->u_in[2]);
  if (!(un < 0.3)) return fail(PSM_ERR_ARG, "|u_in| must be < 0.3 (lattice units)");
  if (lattice->stencil != PSM_D3Q19 && lattice->stencil != PSM_D3Q27) return fail(PSM_ERR_ARG, "bad stencil");
  if (lattice->streaming != PSM_STREAM_AA && lattice->streaming != PSM_STREAM_TWO_GRID)
    return fail(PSM_ERR_ARG, "bad streaming");
  if (lattice->storage < PSM_FP64 || lattice->storage > PSM_BF16_SHIFTED) return fail(PSM_ERR_ARG, "bad storage");
  if (collision->fluid != PSM_BGK && collision->fluid != PSM_TRT && collision->fluid != PSM_CUMULANT)
    return fail(PSM_ERR_ARG, "bad fluid collision");
  if (collision->fluid == PSM_CUMULANT) {
    if (lattice->stencil != PSM_D3Q19) return fail(PSM_ERR_UNSUPPORTED, "the cumulant operator is D3Q19 only");
    for (int k = 0; k < 3; ++k) {
      const double w = collision->cum_omega[k];
      if (!(w == 0.0 || (w > 0.0 && w < 2.0))) return fail(PSM_ERR_ARG, "cum_omega must be 0 (default 1) or in (0, 2)");
    }
  }
  if (!(collision->tau > 0.5) || !std::isfinite(collision->tau)) return fail(PSM_ERR_ARG, "tau must be > 1/2");
  if (collision->fluid == PSM_TRT && !(collision->trt_lambda > 0.0)) return fail(PSM_ERR_ARG, "trt_lambda must be > 0");
  if (collision->solid < PSM_SC1 || collision->solid > PSM_SC3) return fail(PSM_ERR_ARG, "bad solid collision");
  if (collision->weighting != PSM_B_DIRECT && collision->weighting != PSM_B_TAU_WEIGHTED)
    return fail(PSM_ERR_ARG, "bad weighting");

  if (user_bufs) {
    // caller-owned buffers: device memory of the current device, large enough,
    // checked before any launch (a host pointer would fault the kernels)
    const size_t need = (size_t)lattice->stencil * (size_t)grid->nx * (size_t)grid->ny * (size_t)grid->nz *
                        storage_bytes(lattice->storage);
    const int nb = lattice->streaming == PSM_STREAM_TWO_GRID ? 2 : 1;
    for (int b = 0; b < nb; ++b) {
      const int rc = psm::check_device_buffer(user_bufs[b], need, b == 0 ? "PDF buffer 0" : "PDF buffer 1");
      if (rc != PSM_OK) return rc;
    }
  }
  psm_solver* h = new (std::nothrow) psm_solver();
  if (!h) return fail(PSM_ERR_OOM, "host allocation failed");
  h->grid = *grid;
  h->lat = *lattice;
  h->col = *collision;
  h->stream = static_cast<cudaStream_t>(stream);
  h->Q = lattice->stencil;
  h->g.nx = (int)grid->nx;
  h->g.ny = (int)grid->ny;
  h->g.nz = (int)grid->nz;
  h->g.ncell = (long long)grid->nx * grid->ny * grid->nz;
  h->g.bc_z = grid->bc_z;
  h->g.z0 = 0;
  h->tiling = psm::make_tiling(h->g.nx, h->g.ny, h->g.nz);
  fill_ghost(h);

  auto cleanup = [&](int rc) {
    psm_destroy(h);
    return rc;
  };
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "no CUDA device"));
  h->max_blocks = sms * (2048 / psm::PSM_THREADS);
  const size_t bytes = (size_t)h->Q * (size_t)h->g.ncell * storage_bytes(lattice->storage);
  const int nbuf = lattice->streaming == PSM_STREAM_TWO_GRID ? 2 : 1;
  if (user_bufs) {
    h->owns_buf = false;
    for (int b = 0; b < nbuf; ++b) h->buf[b] = user_bufs[b];
  } else {
    for (int b = 0; b < nbuf; ++b) {
      e = cudaMalloc(&h->buf[b], bytes);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "PDF buffer allocation"));
    }
  }
  e = cudaMalloc(&h->d_partials, sizeof(double) * (size_t)h->max_blocks * PSM_MAX_BODIES * 6);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_ticket, sizeof(unsigned int));
  h->cap = 1 << 16;
  if (e == cudaSuccess) e = cudaMalloc(&h->d_series, sizeof(double) * (size_t)h->cap * PSM_MAX_BODIES * 6);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_sum, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(int));
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "scratch allocation"));
  e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "scratch initialisation"));
  // the TMA-staged kernel where the shape allows it
  if (tma_shape(h, h->tma_tiling, h->tma_tiling_odd)) {
    h->tma_ok = true;
    for (int b = 0; b < nbuf; ++b) h->tma_ok = h->tma_ok && encode_maps(h, h->buf[b], h->maps[b], h->tma_tiling);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    h->tma_odd_ok = h->tma_ok && h->tma_tiling.tx == psm::PSM_THREADS &&
                    psm::tma_smem_bytes(h->lat.storage, h->Q, psm::MODE_AA_ODD, h->col.fluid) <= optin;
    h->tma_tg_ok = h->tma_ok && tma_tiling_for(h, psm::MODE_TG, h->tma_tiling_tg) &&
                   psm::tma_smem_bytes(h->lat.storage, h->Q, psm::MODE_TG, h->col.fluid) <= optin;
  }
  e = cudaMemsetAsync(h->d_ticket, 0, sizeof(unsigned int), h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->d_series, 0, sizeof(double) * (size_t)h->cap * PSM_MAX_BODIES * 6, h->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "scratch initialisation"));
  if (!keep) {
    const int rc = import_uniform(h, grid->rho0, grid->u_in);
    if (rc != PSM_OK) return cleanup(rc);
  } else {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "synchronise"));
  }
  *out = h;
  return PSM_OK;
}
}  // namespace

int psm_create(const psm_grid* grid, const psm_lattice* lattice, const psm_collision* collision, void* stream,
               psm_handle* out) {
  return create_impl(grid, lattice, collision, stream, nullptr, false, out);
}

int psm_create_with_buffers(const psm_grid* grid, const psm_lattice* lattice, const psm_collision* collision,
                            void* stream, void* const* buffers, int flags, psm_handle* out) {
  if (!lattice || !buffers) return fail(PSM_ERR_ARG, "psm_create_with_buffers: NULL argument");
  if (flags & ~PSM_BUFFERS_KEEP) return fail(PSM_ERR_ARG, "unknown psm_create_with_buffers flags");
  const int nbuf = lattice->streaming == PSM_STREAM_TWO_GRID ? 2 : 1;
  for (int b = 0; b < nbuf; ++b) {
    if (!buffers[b]) return fail(PSM_ERR_ARG, "PDF buffer %d is NULL", b);
    if (reinterpret_cast<uintptr_t>(buffers[b]) % 16 != 0) return fail(PSM_ERR_ARG, "PDF buffer %d is not 16-byte aligned", b);
  }
  if (nbuf == 2 && buffers[0] == buffers[1]) return fail(PSM_ERR_ARG, "the two PDF buffers must differ");
  return create_impl(grid, lattice, collision, stream, buffers, (flags & PSM_BUFFERS_KEEP) != 0, out);
}

int psm_check_device_buffer(const void* p, int64_t bytes) {
  if (!p) return fail(PSM_ERR_ARG, "psm_check_device_buffer: NULL pointer");
  if (bytes < 0) return fail(PSM_ERR_ARG, "psm_check_device_buffer: negative size");
  return psm::check_device_buffer(p, (size_t)bytes, "buffer");
}

int psm_destroy(psm_handle h) {
  if (!h) return PSM_OK;
  if (h->stream || h->buf[0]) cudaStreamSynchronize(h->stream);
  if (h->owns_buf)
    for (int b = 0; b < 2; ++b) cudaFree(h->buf[b]);
  for (int b = 0; b < PSM_MAX_BODIES; ++b) {
    cudaFree(h->body[b].d_bricks);
    cudaFree(h->body[b].d_occ);
    cudaFree(h->body[b].d_occ8);
  }
  cudaFree(h->d_partials);
  cudaFree(h->d_ticket);
  cudaFree(h->d_series);
  cudaFree(h->d_sum);
  cudaFree(h->d_delta);
  cudaFree(h->d_err);
  for (void* c : h->ckpt) cudaFree(c);
  for (void* c : h->rec_slots) cudaFree(c);
  for (void* c : h->rec_slots2) cudaFree(c);
  cudaFree(h->d_partials2);
  cudaFree(h->d_ticket2);
  if (h->rec_stream) cudaStreamDestroy(h->rec_stream);
  cudaFree(h->d_dyn);
  cudaFree(h->d_dev_bodies);
  cudaFree(h->rec_lam[0]);
  cudaFree(h->rec_lam[1]);
  cudaFree(h->rec_grad);
  delete h;
  return PSM_OK;
}

int psm_init_equilibrium(psm_handle h, double rho, const double u[3]) {
  if (!valid_handle(h) || !u) return fail(PSM_ERR_ARG, "psm_init_equilibrium: NULL argument");
  if (!(rho > 0.0)) return fail(PSM_ERR_ARG, "rho must be > 0");
  return import_uniform(h, rho, u);
}

int psm_set_state(psm_handle h, const double* f) {
  if (!valid_handle(h) || !f) return fail(PSM_ERR_ARG, "psm_set_state: NULL argument");
  const int planes = chunk_planes(h, sizeof(double) * h->Q);
  const size_t plane = (size_t)h->grid.nx * h->grid.ny;
  double* tmp = nullptr;
  PSM_CUDA(cudaMalloc(&tmp, sizeof(double) * h->Q * plane * planes), "state staging allocation");
  int rc = PSM_OK;
  for (int z0 = 0; z0 < h->grid.nz && rc == PSM_OK; z0 += planes) {
    const int z1 = (int)std::min<int64_t>(h->grid.nz, z0 + planes);
    const size_t nchunk = plane * (z1 - z0);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < h->Q && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(tmp + (size_t)i * nchunk, f + (size_t)i * h->g.ncell + (size_t)z0 * plane,
                          sizeof(double) * nchunk, cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "state upload");
      break;
    }
    IoParams p;
    io_base(h, p);
    p.z_begin = z0;
    p.z_end = z1;
    p.f_in = tmp;
    e = psm::launch_import(h->lat.storage, h->Q, p, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "import kernel");
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  return rc;
}

int psm_get_state(psm_handle h, double* f) {
  if (!valid_handle(h) || !f) return fail(PSM_ERR_ARG, "psm_get_state: NULL argument");
  const int planes = chunk_planes(h, sizeof(double) * h->Q);
  const size_t plane = (size_t)h->grid.nx * h->grid.ny;
  double* tmp = nullptr;
  PSM_CUDA(cudaMalloc(&tmp, sizeof(double) * h->Q * plane * planes), "state staging allocation");
  int rc = PSM_OK;
  for (int z0 = 0; z0 < h->grid.nz && rc == PSM_OK; z0 += planes) {
    const int z1 = (int)std::min<int64_t>(h->grid.nz, z0 + planes);
    const size_t nchunk = plane * (z1 - z0);
    IoParams p;
    io_base(h, p);
    p.z_begin = z0;
    p.z_end = z1;
    p.f_out = tmp;
    cudaError_t e = psm::launch_export(h->lat.storage, h->Q, p, h->stream);
    for (int i = 0; i < h->Q && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(f + (size_t)i * h->g.ncell + (size_t)z0 * plane, tmp + (size_t)i * nchunk,
                          sizeof(double) * nchunk, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "state export");
  }
  cudaFree(tmp);
  return rc;
}

int psm_init_equilibrium_field(psm_handle h, const double* rho, const double* u) {
  if (!valid_handle(h) || !rho || !u) return fail(PSM_ERR_ARG, "psm_init_equilibrium_field: NULL argument");
  const int planes = chunk_planes(h, sizeof(double) * 4);
  const size_t plane = (size_t)h->grid.nx * h->grid.ny;
  double* tmp = nullptr;
  PSM_CUDA(cudaMalloc(&tmp, sizeof(double) * 4 * plane * planes), "field staging allocation");
  int rc = PSM_OK;
  for (int z0 = 0; z0 < h->grid.nz && rc == PSM_OK; z0 += planes) {
    const int z1 = (int)std::min<int64_t>(h->grid.nz, z0 + planes);
    const size_t nchunk = plane * (z1 - z0);
    cudaError_t e = cudaMemcpyAsync(tmp, rho + (size_t)z0 * plane, sizeof(double) * nchunk, cudaMemcpyDefault,
                                    h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp + nchunk, u + (size_t)z0 * plane * 3, sizeof(double) * 3 * nchunk, cudaMemcpyDefault,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "field upload");
      break;
    }
    // validate on the host side of the copy: rho > 0 and finite, |u| < 0.3
    std::vector<double> hv(4 * nchunk);
    e = cudaMemcpy(hv.data(), tmp, sizeof(double) * 4 * nchunk, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "field check");
      break;
    }
    for (size_t c = 0; c < nchunk && rc == PSM_OK; ++c) {
      const double r = hv[c], *uc = &hv[nchunk + 3 * c];
      const double un = std::sqrt(uc[0] * uc[0] + uc[1] * uc[1] + uc[2] * uc[2]);
      if (!(r > 0.0) || !std::isfinite(r) || !(un < 0.3))
        rc = fail(PSM_ERR_ARG, "cell %zu: rho must be > 0 and |u| < 0.3", (size_t)z0 * plane + c);
    }
    if (rc != PSM_OK) break;
    IoParams p;
    io_base(h, p);
    p.z_begin = z0;
    p.z_end = z1;
    p.rho_f = tmp;
    p.u_f = tmp + nchunk;
    e = psm::launch_import(h->lat.storage, h->Q, p, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "import kernel");
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  return rc;
}

int psm_get_pdfs(psm_handle h, void* f) {
  if (!valid_handle(h) || !f) return fail(PSM_ERR_ARG, "psm_get_pdfs: NULL argument");
  const size_t b = storage_bytes(h->lat.storage);
  const int planes = chunk_planes(h, b * h->Q);
  const size_t plane = (size_t)h->grid.nx * h->grid.ny;
  char* tmp = nullptr;
  PSM_CUDA(cudaMalloc(&tmp, b * h->Q * plane * planes), "pdf staging allocation");
  int rc = PSM_OK;
  for (int z0 = 0; z0 < h->grid.nz && rc == PSM_OK; z0 += planes) {
    const int z1 = (int)std::min<int64_t>(h->grid.nz, z0 + planes);
    const size_t nchunk = plane * (z1 - z0);
    IoParams p;
    io_base(h, p);
    p.z_begin = z0;
    p.z_end = z1;
    p.f_out_raw = tmp;
    cudaError_t e = psm::launch_export_raw(h->lat.storage, h->Q, p, h->stream);
    for (int i = 0; i < h->Q && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(static_cast<char*>(f) + ((size_t)i * h->g.ncell + (size_t)z0 * plane) * b,
                          tmp + (size_t)i * nchunk * b, b * nchunk, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "pdf export");
  }
  cudaFree(tmp);
  return rc;
}

int psm_get_cells(psm_handle h, const int64_t* cells, int64_t n, double* f) {
  if (!valid_handle(h) || (n > 0 && (!cells || !f))) return fail(PSM_ERR_ARG, "psm_get_cells: NULL argument");
  if (n < 0) return fail(PSM_ERR_ARG, "psm_get_cells: n must be >= 0");
  if (n == 0) return PSM_OK;
  std::vector<long long> hc((size_t)n);
  PSM_CUDA(cudaMemcpy(hc.data(), cells, sizeof(long long) * (size_t)n, cudaMemcpyDefault), "cell list read");
  for (long long c : hc)
    if (c < 0 || c >= h->g.ncell) return fail(PSM_ERR_ARG, "psm_get_cells: cell index %lld out of range", c);
  long long* dc = nullptr;
  double* dout = nullptr;
  PSM_CUDA(cudaMalloc(&dc, sizeof(long long) * (size_t)n), "cell list allocation");
  cudaError_t e = cudaMalloc(&dout, sizeof(double) * (size_t)n * h->Q);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dc, hc.data(), sizeof(long long) * (size_t)n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    IoParams p;
    io_base(h, p);
    switch (h->lat.storage) {
      case PSM_FP64: e = psm::launch_get_cells_fp64(h->Q, p, dc, n, dout, h->stream); break;
      case PSM_FP32: e = psm::launch_get_cells_fp32(h->Q, p, dc, n, dout, h->stream); break;
      case PSM_FP16_SHIFTED: e = psm::launch_get_cells_fp16(h->Q, p, dc, n, dout, h->stream); break;
      default: e = psm::launch_get_cells_bf16(h->Q, p, dc, n, dout, h->stream); break;
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f, dout, sizeof(double) * (size_t)n * h->Q, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(dc);
  cudaFree(dout);
  if (e != cudaSuccess) return cuda_fail(e, "psm_get_cells");
  return PSM_OK;
}

int psm_get_macroscopic(psm_handle h, double* rho, double* u) {
  if (!valid_handle(h) || !rho || !u) return fail(PSM_ERR_ARG, "psm_get_macroscopic: NULL argument");
  const int planes = chunk_planes(h, sizeof(double) * 4);
  const size_t plane = (size_t)h->grid.nx * h->grid.ny;
  double* tmp = nullptr;
  PSM_CUDA(cudaMalloc(&tmp, sizeof(double) * 4 * plane * planes), "macroscopic staging allocation");
  int rc = PSM_OK;
  for (int z0 = 0; z0 < h->grid.nz && rc == PSM_OK; z0 += planes) {
    const int z1 = (int)std::min<int64_t>(h->grid.nz, z0 + planes);
    const size_t nchunk = plane * (z1 - z0);
    IoParams p;
    io_base(h, p);
    p.z_begin = z0;
    p.z_end = z1;
    p.rho_out = tmp;
    p.u_out = tmp + nchunk;
    cudaError_t e = psm::launch_macro(h->lat.storage, h->Q, p, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rho + (size_t)z0 * plane, tmp, sizeof(double) * nchunk, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(u + 3 * (size_t)z0 * plane, tmp + nchunk, sizeof(double) * 3 * nchunk, cudaMemcpyDefault,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "macroscopic export");
  }
  cudaFree(tmp);
  return rc;
}

int psm_get_eps(psm_handle h, float* eps) {
  if (!valid_handle(h) || !eps) return fail(PSM_ERR_ARG, "psm_get_eps: NULL argument");
  const int planes = chunk_planes(h, sizeof(float));
  const size_t plane = (size_t)h->grid.nx * h->grid.ny;
  float* tmp = nullptr;
  PSM_CUDA(cudaMalloc(&tmp, sizeof(float) * plane * planes), "eps staging allocation");
  int rc = PSM_OK;
  for (int z0 = 0; z0 < h->grid.nz && rc == PSM_OK; z0 += planes) {
    const int z1 = (int)std::min<int64_t>(h->grid.nz, z0 + planes);
    psm::RemapParams p;
    std::memset(&p, 0, sizeof p);
    p.g = h->g;
    p.t = h->tiling;
    p.nbodies = h->nbodies;
    for (int b = 0; b < h->nbodies; ++b) p.body[b] = dev_body(h, b, h->step);
    if (h->free_mask) {
      // two-way coupled bodies: their pose of this step lives on the device
      cudaError_t e0 = cudaStreamSynchronize(h->stream);
      for (int b = 0; b < h->nbodies && e0 == cudaSuccess; ++b)
        if ((h->free_mask >> b) & 1u) e0 = cudaMemcpy(&p.body[b], h->d_dev_bodies + b, sizeof(DevBody), cudaMemcpyDeviceToHost);
      if (e0 != cudaSuccess) {
        rc = cuda_fail(e0, "body state read");
        break;
      }
    }
    p.z_begin = z0;
    p.z_end = z1;
    p.eps_out = tmp;
    cudaError_t e = psm::launch_remap(p, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(eps + (size_t)z0 * plane, tmp, sizeof(float) * plane * (z1 - z0), cudaMemcpyDefault,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "eps export");
  }
  cudaFree(tmp);
  return rc;
}

int psm_set_geometry(psm_handle h, int body, const psm_geom_field* field, const double Q0[9], const double R0[3],
                     const double omega[3], const double v[3]) {
  if (!valid_handle(h) || !field || !Q0 || !R0 || !omega || !v)
    return fail(PSM_ERR_ARG, "psm_set_geometry: NULL argument");
  if (body < 0 || body >= PSM_MAX_BODIES || body > h->nbodies)
    return fail(PSM_ERR_ARG, "body id %d: bodies are numbered contiguously from 0 (max %d)", body, PSM_MAX_BODIES);
  if (field->s < 0 || field->s > 3) return fail(PSM_ERR_ARG, "super-sampling depth s must be 0..3");
  if (field->gx < 1 || field->gy < 1 || field->gz < 1 || field->gx > (1 << 20) || field->gy > (1 << 20) ||
      field->gz > (1 << 20))
    return fail(PSM_ERR_ARG, "geometry field dims must be in 1..2^20");
  if (!field->bricks) return fail(PSM_ERR_ARG, "geometry field has no bricks");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(field->lo[k]) || !std::isfinite(R0[k]) || !std::isfinite(omega[k]) || !std::isfinite(v[k]))
      return fail(PSM_ERR_ARG, "non-finite body parameter");
  const int wpb = field->s == 3 ? 8 : 1;
  const size_t words = (size_t)field->gx * field->gy * field->gz * wpb;
  HostBody& b = h->body[body];
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronise before geometry upload");
  cudaFree(b.d_bricks);
  b.d_bricks = nullptr;
  PSM_CUDA(cudaMalloc(&b.d_bricks, words * sizeof(unsigned long long)), "geometry field allocation");
  PSM_CUDA(cudaMemcpy(b.d_bricks, field->bricks, words * sizeof(unsigned long long), cudaMemcpyDefault),
           "geometry field upload");
  cudaFree(b.d_occ);
  b.d_occ = nullptr;
  const size_t nocc = (size_t)(field->gx + 1) * (field->gy + 1) * (field->gz + 1);
  PSM_CUDA(cudaMalloc(&b.d_occ, nocc), "geometry occupancy allocation");
  PSM_CUDA(psm::launch_occupancy(b.d_bricks, (int)field->gx, (int)field->gy, (int)field->gz, wpb, b.d_occ, h->stream),
           "geometry occupancy kernel");
  cudaFree(b.d_occ8);
  b.d_occ8 = nullptr;
  {
    const int ox = (int)field->gx + 1, oy = (int)field->gy + 1, oz = (int)field->gz + 1;
    const size_t nb8 = (size_t)((ox + 7) / 8) * ((oy + 7) / 8) * ((oz + 7) / 8);
    const size_t words8 = (nb8 + 31) / 32;
    PSM_CUDA(cudaMalloc(&b.d_occ8, words8 * sizeof(unsigned)), "geometry block occupancy allocation");
    PSM_CUDA(cudaMemsetAsync(b.d_occ8, 0, words8 * sizeof(unsigned), h->stream), "geometry block occupancy");
    PSM_CUDA(psm::launch_occupancy8(b.d_occ, ox, oy, oz, b.d_occ8, h->stream), "geometry block occupancy kernel");
  }
  PSM_CUDA(cudaStreamSynchronize(h->stream), "geometry occupancy");
  b.gx = field->gx;
  b.gy = field->gy;
  b.gz = field->gz;
  b.s = field->s;
  b.wpb = wpb;
  for (int k = 0; k < 3; ++k) {
    b.lo[k] = field->lo[k];
    b.R0[k] = R0[k];
    b.omega[k] = omega[k];
    b.us_omega[k] = omega[k];
    b.v[k] = v[k];
  }
  for (int k = 0; k < 9; ++k) b.Q0[k] = Q0[k];
  h->free_mask &= ~(1u << body);  // prescribed motion again
  if (body == h->nbodies) h->nbodies++;
  return PSM_OK;
}

int psm_set_us_omega(psm_handle h, int body, const double omega[3]) {
  if (!valid_handle(h) || !omega) return fail(PSM_ERR_ARG, "psm_set_us_omega: NULL argument");
  if (body < 0 || body >= h->nbodies) return fail(PSM_ERR_ARG, "no body %d", body);
  if ((h->free_mask >> body) & 1u) return fail(PSM_ERR_STATE, "body %d moves under the fluid's load", body);
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(omega[k])) return fail(PSM_ERR_ARG, "omega must be finite");
  for (int k = 0; k < 3; ++k) h->body[body].us_omega[k] = omega[k];
  return PSM_OK;
}

int psm_num_bodies(psm_handle h, int* out) {
  if (!valid_handle(h) || !out) return fail(PSM_ERR_ARG, "psm_num_bodies: NULL argument");
  *out = h->nbodies;
  return PSM_OK;
}

int psm_step(psm_handle h, int n) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_step: NULL handle");
  if (n < 0) return fail(PSM_ERR_ARG, "psm_step: n must be >= 0");
  StepParams p;
  std::memset(&p, 0, sizeof p);
  const bool use_tma = h->tma_ok && h->variant != PSM_KERNEL_PLAIN;
  p.g = h->g;
  p.t = use_tma ? h->tma_tiling : h->tiling;
  fill_consts<float>(h, p.cf);
  fill_consts<double>(h, p.cd);
  p.fluid = h->col.fluid;
  p.solid = h->col.solid;
  p.weighting = h->col.weighting;
  p.nbodies = h->nbodies;
  p.delta = h->d_delta;
  p.partials = h->d_partials;
  p.ticket = h->d_ticket;
  p.err = h->d_err;
  for (int k = 0; k < n; ++k) {
    if (h->recording && (h->step - h->rec_n0) % h->rec_K == 0 &&
        (int64_t)h->ckpt.size() == (h->step - h->rec_n0) / h->rec_K) {
      const int rc = take_checkpoint(h);
      if (rc != PSM_OK) return rc;
    }
    for (int b = 0; b < h->nbodies; ++b) p.body[b] = dev_body(h, b, h->step);
    p.ft_out = h->d_series + (size_t)(h->step % h->cap) * PSM_MAX_BODIES * 6;
    int mode, src;
    if (h->lat.streaming == PSM_STREAM_TWO_GRID) {
      mode = psm::MODE_TG;
      src = h->cur;
      p.f = h->buf[h->cur];
      p.f_dst = h->buf[h->cur ^ 1];
    } else {
      mode = (h->step & 1) ? psm::MODE_AA_ODD : psm::MODE_AA_EVEN;
      src = 0;
      p.f = h->buf[0];
      p.f_dst = nullptr;
    }
    psm::set_slots(p, h->lat.storage, h->Q);
    p.free_mask = h->free_mask;
    p.dbody = h->d_dev_bodies;
    // the AA odd step runs with plain loads unless its TMA variant applies
    const bool tma_now = use_tma && (mode != psm::MODE_AA_ODD ||
                                     (h->tma_odd_ok && (h->variant == PSM_KERNEL_TMA || !PSM_AA_ODD_PLAIN)));
    p.t = !tma_now ? h->tiling : (mode == psm::MODE_AA_ODD ? h->tma_tiling_odd : h->tma_tiling);
    psm::TmaMaps tm;
    if (tma_now) {
      const int dsti = h->lat.streaming == PSM_STREAM_TWO_GRID ? (src ^ 1) : 0;
      tm.tile = h->maps[src].tile;
      tm.row1 = h->maps[src].row1;
      tm.dstw = h->maps[dsti].warpq;
    }
    cudaError_t e = tma_now ? psm::launch_step_tma(h->lat.storage, h->Q, mode, p, tm, h->stream)
                            : psm::launch_step(h->lat.storage, h->Q, mode, p, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    if (h->free_mask) {
      e = psm::launch_body_update(h->d_dyn, h->d_dev_bodies, p.ft_out, h->free_mask, h->nbodies, (int)h->grid.nx,
                                  (int)h->grid.ny, (int)h->grid.nz, h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "body update launch");
    }
    if (h->lat.streaming == PSM_STREAM_TWO_GRID) h->cur ^= 1;
    h->step++;
  }
  return PSM_OK;
}

int psm_set_eps_delta(psm_handle h, const float* delta) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_set_eps_delta: NULL handle");
  PSM_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  if (!delta) {
    cudaFree(h->d_delta);
    h->d_delta = nullptr;
    return PSM_OK;
  }
  if (!h->d_delta) PSM_CUDA(cudaMalloc(&h->d_delta, sizeof(float) * (size_t)h->g.ncell), "delta allocation");
  PSM_CUDA(cudaMemcpy(h->d_delta, delta, sizeof(float) * (size_t)h->g.ncell, cudaMemcpyDefault), "delta upload");
  return PSM_OK;
}

// Buffers of psm_backward, allocated when recording starts (a one-time cost
// outside the backward sweep) and kept by the handle: K - 1 recompute states
// with their tensor maps, two adjoint fields, the gradient accumulator.
// The second recompute set of psm_backward (K - 1 states, their tensor maps,
// the recompute stream and its reduction scratch), allocated only while at
// least a sixteenth of the device memory stays free; without it psm_backward
// recomputes and sweeps each segment in turn on the solver's stream.
static void ensure_second_recompute_set(psm_solver* h, int K) {
  for (void* c : h->rec_slots2) cudaFree(c);
  h->rec_slots2.clear();
  h->rec_maps2.clear();
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if ((size_t)(K - 1) * state_bytes(h) + total_b / 16 > free_b) return;
  std::vector<void*> slots((size_t)K, nullptr);
  std::vector<BufMaps> maps((size_t)K, BufMaps{});
  bool ok = true;
  for (int k = 1; k < K && ok; ++k) {
    ok = cudaMalloc(&slots[k], state_bytes(h)) == cudaSuccess;
    if (ok && h->tma_tg_ok) ok = encode_maps(h, slots[k], maps[k], h->tma_tiling_tg);
  }
  if (ok && !h->rec_stream) ok = cudaStreamCreateWithFlags(&h->rec_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (ok && !h->d_partials2)
    ok = cudaMalloc(&h->d_partials2, sizeof(double) * (size_t)h->max_blocks * PSM_MAX_BODIES * 6) == cudaSuccess;
  if (ok && !h->d_ticket2) {
    ok = cudaMalloc(&h->d_ticket2, sizeof(unsigned int)) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(h->d_ticket2, 0, sizeof(unsigned int), h->stream) == cudaSuccess;
    if (!ok) {
      cudaFree(h->d_ticket2);
      h->d_ticket2 = nullptr;
    }
  }
  if (!ok) {
    cudaGetLastError();  // an allocation that failed is not an error of the call
    for (void* c : slots) cudaFree(c);
    return;
  }
  h->rec_slots2 = slots;
  h->rec_maps2 = maps;
}

int ensure_backward_buffers(psm_solver* h, int K, bool second) {
  const size_t ncell = (size_t)h->g.ncell;
  const size_t tb = h->lat.storage == PSM_FP64 ? 8 : 4;
  cudaError_t e = cudaSuccess;
  if ((int)h->rec_slots.size() != K) {
    PSM_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
    for (void* c : h->rec_slots) cudaFree(c);
    h->rec_slots.assign((size_t)K, nullptr);
    h->rec_maps.assign((size_t)K, BufMaps{});
    for (int k = 1; k < K && e == cudaSuccess; ++k) {
      e = cudaMalloc(&h->rec_slots[k], state_bytes(h));
      if (e == cudaSuccess && h->tma_tg_ok && !encode_maps(h, h->rec_slots[k], h->rec_maps[k], h->tma_tiling_tg))
        e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) {
      for (void* c : h->rec_slots) cudaFree(c);
      h->rec_slots.clear();
      h->rec_maps.clear();
      return cuda_fail(e, "backward recompute buffers");
    }
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    if (!h->rec_lam[k]) e = cudaMalloc(&h->rec_lam[k], (size_t)h->Q * ncell * tb);
  if (e == cudaSuccess && !h->rec_grad) e = cudaMalloc((void**)&h->rec_grad, ncell * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "backward buffers");
  if (!second) {
    for (void* c : h->rec_slots2) cudaFree(c);
    h->rec_slots2.clear();
    h->rec_maps2.clear();
  } else if (K > 1 && h->rec_slots2.size() != (size_t)K) {
    ensure_second_recompute_set(h, K);
  }
  return PSM_OK;
}

int psm_record(psm_handle h, int K, int flags) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_record: NULL handle");
  drop_checkpoints(h);
  h->recording = false;
  if (K == 0) return PSM_OK;
  if (K < 1) return fail(PSM_ERR_ARG, "checkpoint interval K must be >= 1 (0 stops recording)");
  if (h->lat.streaming == PSM_STREAM_AA && ((K & 1) || (h->step & 1)))
    return fail(PSM_ERR_ARG, "AA streaming: record from an even step with an even K (checkpoints need the "
                             "natural layout)");
  if (flags & ~(PSM_RECORD_INIT_FROM_INFLOW | PSM_RECORD_SEQUENTIAL)) return fail(PSM_ERR_ARG, "unknown record flags");
  if (h->col.fluid == PSM_CUMULANT)
    return fail(PSM_ERR_UNSUPPORTED, "psm_backward supports BGK and TRT (no adjoint of the cumulant operator)");
  if (h->slab) return fail(PSM_ERR_UNSUPPORTED, "psm_backward of a z-slab (the adjoint is not decomposed)");
  if (h->free_mask)
    return fail(PSM_ERR_STATE, "psm_backward supports prescribed motion only (two-way coupled bodies attached)");
  {
    const int rc = ensure_backward_buffers(h, K, !(flags & PSM_RECORD_SEQUENTIAL));
    if (rc != PSM_OK) return rc;
  }
  h->rec_K = K;
  h->rec_flags = flags;
  h->rec_n0 = h->step;
  h->recording = true;
  return take_checkpoint(h);
}

int psm_backward(psm_handle h, const double* dJ_dFT, double* grad_eps, double* grad_omega, double* grad_uin) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_backward: NULL handle");
  if (!h->recording) return fail(PSM_ERR_STATE, "psm_backward needs a forward run recorded with psm_record");
  const int64_t N = h->step - h->rec_n0;
  if (N < 1) return fail(PSM_ERR_STATE, "no step recorded since psm_record");
  const int K = h->rec_K;
  const int64_t M = (N + K - 1) / K;
  if ((int64_t)h->ckpt.size() < M) return fail(PSM_ERR_STATE, "checkpoints missing");
  const int nb = h->nbodies;
  const int ncomp = nb * 3 + 3;
  const size_t ncell = (size_t)h->g.ncell;
  const size_t tb = h->lat.storage == PSM_FP64 ? 8 : 4;
  cudaStream_t st = h->stream;
  // weights of J on the force/torque series
  std::vector<double> w((size_t)N * nb * 6, 0.0);
  if (dJ_dFT) {
    PSM_CUDA(cudaMemcpy(w.data(), dJ_dFT, sizeof(double) * w.size(), cudaMemcpyDefault), "weights upload");
  } else {
    if (nb < 1) return fail(PSM_ERR_STATE, "default functional (mean torque) needs a body");
    for (int64_t n = 0; n < N; ++n) w[(size_t)n * nb * 6 + 5] = 1.0 / (double)N;
  }
  // recompute buffers, adjoint fields and gradient accumulator: allocated by
  // psm_record (ensure_backward_buffers)
  {
    const int rc = ensure_backward_buffers(h, K, !(h->rec_flags & PSM_RECORD_SEQUENTIAL));
    if (rc != PSM_OK) return rc;
  }
  // one or two recompute sets (set 1: the segment before the current one,
  // recomputed on the recompute stream while the adjoint sweeps the current)
  const bool overlap =
      !(h->rec_flags & PSM_RECORD_SEQUENTIAL) && M > 1 && h->rec_slots2.size() == (size_t)K && h->rec_stream;
  std::vector<void*> slots[2] = {h->rec_slots, h->rec_slots2};
  std::vector<BufMaps> smaps[2] = {h->rec_maps, h->rec_maps2};
  const bool tma_rec = h->tma_tg_ok && h->variant != PSM_KERNEL_PLAIN;
  void* lam0 = h->rec_lam[0];
  void* lam1 = h->rec_lam[1];
  double* grad = h->rec_grad;
  // small scratch (stream ordered): the weights and the per-step accumulators
  double *wdev = nullptr, *acc = nullptr, *ftscratch = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&wdev, sizeof(double) * w.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&acc, sizeof(double) * (size_t)(N + 1) * ncomp, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&ftscratch, sizeof(double) * PSM_MAX_BODIES * 6, st);
  auto release = [&]() {
    cudaFreeAsync(wdev, st);
    cudaFreeAsync(acc, st);
    cudaFreeAsync(ftscratch, st);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "backward scratch allocation");
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(wdev, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(lam0, 0, (size_t)h->Q * ncell * tb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, ncell * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)(N + 1) * ncomp, st);

  // step parameters for the recompute (two-grid; TMA-staged where the shape
  // allows, like the forward) and the adjoint
  StepParams sp;
  std::memset(&sp, 0, sizeof sp);
  sp.g = h->g;
  sp.t = tma_rec ? h->tma_tiling_tg : h->tiling;
  fill_consts<float>(h, sp.cf);
  fill_consts<double>(h, sp.cd);
  sp.fluid = h->col.fluid;
  sp.solid = h->col.solid;
  sp.weighting = h->col.weighting;
  sp.nbodies = nb;
  sp.delta = h->d_delta;
  sp.partials = h->d_partials;
  sp.ticket = h->d_ticket;
  sp.ft_out = ftscratch;
  sp.err = h->d_err;
  psm::AdjParams ap;
  std::memset(&ap, 0, sizeof ap);
  ap.g = h->g;
  ap.t = h->tiling;
  ap.grad = grad;
  ap.trt = sp.fluid == PSM_TRT ? 1 : 0;
  ap.solid = sp.solid;
  ap.weighting = sp.weighting;
  ap.nbodies = nb;
  ap.delta = h->d_delta;
  ap.partials = h->d_partials;
  ap.ticket = h->d_ticket;
  ap.cf = sp.cf;
  ap.cd = sp.cd;
  {
    // d g_i / d u_in = w_i rho0 (3 c_i + 9 (c_i . u_in) c_i - 3 u_in)
    const double* u = h->grid.u_in;
    for (int i = 0; i < h->Q; ++i) {
      const double wi = h->Q == 19 ? psm::lat_w<19>(i) : psm::lat_w<27>(i);
      const double c[3] = {(double)psm::lat_cx(i), (double)psm::lat_cy(i), (double)psm::lat_cz(i)};
      const double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
      for (int k = 0; k < 3; ++k) {
        ap.dghost[i][k] = wi * h->grid.rho0 * (3.0 * c[k] + 9.0 * cu * c[k] - 3.0 * u[k]);
        ap.dghostf[i][k] = (float)ap.dghost[i][k];
      }
    }
  }
  void* la = lam0;  // lambda^{n+1}
  void* lb = lam1;  // lambda^n
  cudaStream_t rs = overlap ? h->rec_stream : st;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // start, recomputed[2], swept[2]
  bool swept_pending[2] = {false, false};
  if (overlap) {
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    // the recompute stream starts after everything queued on the solver's stream
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, ev[0], 0);
  }
  StepParams rp = sp;  // the recompute's own reduction scratch when it runs beside the adjoint
  if (overlap) {
    rp.partials = h->d_partials2;
    rp.ticket = h->d_ticket2;
  }
  // recompute f^{ns+1} .. f^{ne-1} of segment m into set q
  auto recompute = [&](int64_t m, int q) {
    if (e != cudaSuccess) return;
    if (overlap && swept_pending[q]) e = cudaStreamWaitEvent(rs, ev[3 + q], 0);  // set q read by the adjoint
    const int64_t ns = h->rec_n0 + m * K;
    const int64_t ne = std::min<int64_t>(ns + K, h->step);
    std::vector<void*>& sl = slots[q];
    std::vector<BufMaps>& sm = smaps[q];
    sl[0] = h->ckpt[(size_t)m];
    if (e == cudaSuccess && tma_rec && ne - ns > 1 && !encode_maps(h, sl[0], sm[0], h->tma_tiling_tg))
      e = cudaErrorInvalidValue;
    for (int64_t n = ns; n + 1 < ne && e == cudaSuccess; ++n) {
      for (int b = 0; b < nb; ++b) rp.body[b] = dev_body(h, b, n);
      const size_t a = (size_t)(n - ns), c = a + 1;
      rp.f = sl[a];
      rp.f_dst = sl[c];
      psm::set_slots(rp, h->lat.storage, h->Q);
      if (tma_rec) {
        psm::TmaMaps tm;
        tm.tile = sm[a].tile;
        tm.row1 = sm[a].row1;
        tm.dstw = sm[c].warpq;
        e = psm::launch_step_tma(h->lat.storage, h->Q, psm::MODE_TG, rp, tm, rs);
      } else {
        e = psm::launch_step(h->lat.storage, h->Q, psm::MODE_TG, rp, rs);
      }
    }
    if (overlap && e == cudaSuccess) e = cudaEventRecord(ev[1 + q], rs);
  };
  // adjoint steps ne-1 .. ns of segment m from set q
  auto sweep = [&](int64_t m, int q) {
    if (e != cudaSuccess) return;
    if (overlap) e = cudaStreamWaitEvent(st, ev[1 + q], 0);
    const int64_t ns = h->rec_n0 + m * K;
    const int64_t ne = std::min<int64_t>(ns + K, h->step);
    for (int64_t n = ne - 1; n >= ns && e == cudaSuccess; --n) {
      for (int b = 0; b < nb; ++b) ap.body[b] = dev_body(h, b, n);
      ap.f = slots[q][(size_t)(n - ns)];
      ap.lam_in = la;
      ap.lam_out = lb;
      {
        const size_t fb = storage_bytes(h->lat.storage);
        for (int i = 0; i < 27; ++i) {
          const bool in = i < h->Q;
          ap.f_slot[i] = in ? static_cast<const char*>(ap.f) + (size_t)i * ncell * fb : nullptr;
          ap.lin_slot[i] = in ? static_cast<const char*>(la) + (size_t)i * ncell * tb : nullptr;
          ap.lout_slot[i] = in ? static_cast<char*>(lb) + (size_t)i * ncell * tb : nullptr;
        }
      }
      ap.w = wdev + (size_t)(n - h->rec_n0) * nb * 6;
      ap.acc_out = acc + (size_t)(n - h->rec_n0) * ncomp;
      e = launch_adjoint(h->lat.storage, h->Q, ap.trt, ap, st);
      std::swap(la, lb);
    }
    if (overlap && e == cudaSuccess) {
      e = cudaEventRecord(ev[3 + q], st);
      swept_pending[q] = true;
    }
  };
  if (overlap) {
    // segment m in set (M - 1 - m) mod 2; segment m - 1 is recomputed while m is swept
    recompute(M - 1, 0);
    for (int64_t m = M - 1; m >= 0; --m) {
      const int q = (int)((M - 1 - m) & 1);
      if (m >= 1) recompute(m - 1, q ^ 1);
      sweep(m, q);
    }
  } else {
    for (int64_t m = M - 1; m >= 0; --m) {
      recompute(m, 0);
      sweep(m, 0);
    }
  }
  if (overlap) {
    // whatever happened, the solver's stream ends after the recompute stream
    cudaEventRecord(ev[0], rs);
    cudaStreamWaitEvent(st, ev[0], 0);
    for (int k = 0; k < 5; ++k)
      if (ev[k]) cudaEventDestroy(ev[k]);
  }
  if (e == cudaSuccess && (h->rec_flags & PSM_RECORD_INIT_FROM_INFLOW)) {
    ap.lam_in = la;  // lambda^{n0}
    ap.acc_out = acc + (size_t)N * ncomp + nb * 3;
    e = launch_adjoint_init(h->lat.storage, h->Q, ap, h->max_blocks, st);
  }
  std::vector<double> acc_h((size_t)(N + 1) * ncomp);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(acc_h.data(), acc, sizeof(double) * acc_h.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grad_eps)
    e = cudaMemcpyAsync(grad_eps, grad, sizeof(double) * ncell, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) return cuda_fail(e, "backward pass");
  {
    const int rc = check_err(h);
    if (rc != PSM_OK) return rc;
  }
  // scalar gradients: sum the per-step FP64 partials in step order
  std::vector<double> gw((size_t)nb * 3, 0.0), gu(3, 0.0);
  bool finite = true;
  for (int64_t n = 0; n <= N; ++n) {
    const double* a = acc_h.data() + (size_t)n * ncomp;
    for (int k = 0; k < nb * 3; ++k) gw[k] += a[k];
    for (int k = 0; k < 3; ++k) gu[k] += a[nb * 3 + k];
  }
  for (double v : gw) finite = finite && std::isfinite(v);
  for (double v : gu) finite = finite && std::isfinite(v);
  if (grad_omega) std::memcpy(grad_omega, gw.data(), sizeof(double) * gw.size());
  if (grad_uin) std::memcpy(grad_uin, gu.data(), sizeof(double) * 3);
  if (!finite) return fail(PSM_ERR_NONFINITE, "gradient holds NaN or Inf");
  return PSM_OK;
}

int psm_tma_layout(int storage, int stencil, int mode, int fluid, int* out) {
  if (!out) return fail(PSM_ERR_ARG, "psm_tma_layout: NULL out");
  if (storage < PSM_FP64 || storage > PSM_BF16_SHIFTED) return fail(PSM_ERR_ARG, "bad storage");
  if (stencil != PSM_D3Q19 && stencil != PSM_D3Q27) return fail(PSM_ERR_ARG, "bad stencil");
  if (mode < psm::MODE_TG || mode > psm::MODE_AA_ODD) return fail(PSM_ERR_ARG, "bad mode");
  if (fluid != PSM_BGK && fluid != PSM_TRT && fluid != PSM_CUMULANT) return fail(PSM_ERR_ARG, "bad fluid collision");
  if (fluid == PSM_CUMULANT && stencil != PSM_D3Q19)
    return fail(PSM_ERR_UNSUPPORTED, "the cumulant operator is D3Q19 only");
  switch (storage) {
    case PSM_FP64: psm::tma_layout_fp64(stencil, mode, fluid, out); break;
    case PSM_FP32: psm::tma_layout_fp32(stencil, mode, fluid, out); break;
    case PSM_FP16_SHIFTED: psm::tma_layout_fp16(stencil, mode, fluid, out); break;
    default: psm::tma_layout_bf16(stencil, mode, fluid, out); break;
  }
  return PSM_OK;
}

int psm_set_kernel_variant(psm_handle h, int variant) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_set_kernel_variant: NULL handle");
  if (variant != PSM_KERNEL_AUTO && variant != PSM_KERNEL_PLAIN && variant != PSM_KERNEL_TMA)
    return fail(PSM_ERR_ARG, "unknown kernel variant %d", variant);
  if (variant == PSM_KERNEL_TMA && !h->tma_ok)
    return fail(PSM_ERR_UNSUPPORTED, "the TMA-staged kernel does not support this grid shape / storage");
  h->variant = variant;
  return PSM_OK;
}

int psm_kernel_variant(psm_handle h, int* out) {
  if (!valid_handle(h) || !out) return fail(PSM_ERR_ARG, "psm_kernel_variant: NULL argument");
  *out = (h->tma_ok && h->variant != PSM_KERNEL_PLAIN) ? PSM_KERNEL_TMA : PSM_KERNEL_PLAIN;
  return PSM_OK;
}

int psm_step_count(psm_handle h, int64_t* out) {
  if (!valid_handle(h) || !out) return fail(PSM_ERR_ARG, "psm_step_count: NULL argument");
  *out = h->step;
  return PSM_OK;
}

int psm_series_capacity(psm_handle h, int64_t* out) {
  if (!valid_handle(h) || !out) return fail(PSM_ERR_ARG, "psm_series_capacity: NULL argument");
  *out = h->cap;
  return PSM_OK;
}

int psm_force_torque(psm_handle h, int body, int64_t step_from, int64_t count, double* out) {
  if (!valid_handle(h) || (!out && count > 0)) return fail(PSM_ERR_ARG, "psm_force_torque: NULL argument");
  if (body < 0 || body >= h->nbodies) return fail(PSM_ERR_ARG, "no body %d", body);
  if (count < 0 || step_from < 0 || step_from + count > h->step)
    return fail(PSM_ERR_ARG, "steps [%lld, %lld) not yet computed (step count %lld)", (long long)step_from,
                (long long)(step_from + count), (long long)h->step);
  if (step_from < h->step - h->cap)
    return fail(PSM_ERR_ARG, "step %lld is older than the kept series (%lld steps)", (long long)step_from,
                (long long)h->cap);
  PSM_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  {
    const int rc = check_err(h);
    if (rc != PSM_OK) return rc;
  }
  const size_t row = PSM_MAX_BODIES * 6;
  std::vector<double> tmp(row);
  bool finite = true;
  // copy in at most two contiguous runs of the ring buffer
  int64_t done = 0;
  std::vector<double> rows;
  while (done < count) {
    const int64_t s = step_from + done;
    const int64_t slot = s % h->cap;
    int64_t run = std::min<int64_t>(count - done, h->cap - slot);
    rows.resize((size_t)run * row);
    PSM_CUDA(cudaMemcpy(rows.data(), h->d_series + (size_t)slot * row, sizeof(double) * row * run,
                        cudaMemcpyDeviceToHost),
             "force/torque download");
    for (int64_t r = 0; r < run; ++r)
      for (int k = 0; k < 6; ++k) {
        const double v = rows[(size_t)r * row + body * 6 + k];
        out[(done + r) * 6 + k] = v;
        finite = finite && std::isfinite(v);
      }
    done += run;
  }
  if (!finite) return fail(PSM_ERR_NONFINITE, "force/torque series holds NaN or Inf");
  return PSM_OK;
}

int psm_force_torque_raw(psm_handle h, int body, int64_t step_from, int64_t count, double* out) {
  const int rc = psm_force_torque(h, body, step_from, count, out);
  if (rc != PSM_OK) return rc;
  for (int64_t k = 0; k < count * 6; ++k) out[k] = -out[k];
  return PSM_OK;
}

int psm_set_remap(psm_handle h, int every_step) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_set_remap: NULL handle");
  if (every_step != 0 && every_step != 1) return fail(PSM_ERR_ARG, "psm_set_remap: every_step must be 0 or 1");
  if (h->recording) return fail(PSM_ERR_STATE, "psm_set_remap while recording for psm_backward");
  if (h->free_mask) return fail(PSM_ERR_STATE, "psm_set_remap with two-way coupled bodies");
  if (!every_step && !h->remap_frozen) h->frozen_step = h->step;
  h->remap_frozen = !every_step;
  return PSM_OK;
}

int psm_set_z_offset(psm_handle h, int64_t z0) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_set_z_offset: NULL handle");
  if (z0 < 0 || z0 + h->grid.nz > (int64_t)(1 << 30)) return fail(PSM_ERR_ARG, "z0 must be in [0, 2^30 - nz]");
  if (h->recording) return fail(PSM_ERR_STATE, "psm_set_z_offset while recording for psm_backward");
  if (h->free_mask) return fail(PSM_ERR_STATE, "psm_set_z_offset with two-way coupled bodies");
  h->g.z0 = (int)z0;
  h->slab = true;
  return PSM_OK;
}

int psm_slot_plane(psm_handle h, int slot, int z, void** out) {
  if (!valid_handle(h) || !out) return fail(PSM_ERR_ARG, "psm_slot_plane: NULL argument");
  if (slot < 0 || slot >= h->Q) return fail(PSM_ERR_ARG, "slot %d out of range (Q = %d)", slot, h->Q);
  if (z < 0 || z >= h->grid.nz) return fail(PSM_ERR_ARG, "plane %d out of range (nz = %d)", z, (int)h->grid.nz);
  *out = slot_plane_addr(h, slot, z);
  return PSM_OK;
}

int psm_fill_slot_plane(psm_handle h, int slot, int z, int dir) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_fill_slot_plane: NULL handle");
  if (slot < 0 || slot >= h->Q) return fail(PSM_ERR_ARG, "slot %d out of range (Q = %d)", slot, h->Q);
  if (dir < 0 || dir >= h->Q) return fail(PSM_ERR_ARG, "direction %d out of range (Q = %d)", dir, h->Q);
  if (z < 0 || z >= h->grid.nz) return fail(PSM_ERR_ARG, "plane %d out of range (nz = %d)", z, (int)h->grid.nz);
  void* dst = slot_plane_addr(h, slot, z);
  const long long n = (long long)h->grid.nx * h->grid.ny;
  const int blocks = (int)std::min<long long>((n + psm::PSM_THREADS - 1) / psm::PSM_THREADS, 1024);
  const double v = h->ghost[dir];
  switch (h->lat.storage) {
    case PSM_FP64: psm::k_fill_plane<double><<<blocks, psm::PSM_THREADS, 0, h->stream>>>((double*)dst, n, v); break;
    case PSM_FP32: psm::k_fill_plane<float><<<blocks, psm::PSM_THREADS, 0, h->stream>>>((float*)dst, n, v); break;
    case PSM_FP16_SHIFTED: psm::k_fill_plane<__half><<<blocks, psm::PSM_THREADS, 0, h->stream>>>((__half*)dst, n, v); break;
    default: psm::k_fill_plane<__nv_bfloat16><<<blocks, psm::PSM_THREADS, 0, h->stream>>>((__nv_bfloat16*)dst, n, v); break;
  }
  PSM_CUDA(cudaGetLastError(), "plane fill launch");
  return PSM_OK;
}

int psm_set_body_dynamics(psm_handle h, int body, const psm_body_dynamics* dyn) {
  if (!valid_handle(h) || !dyn) return fail(PSM_ERR_ARG, "psm_set_body_dynamics: NULL argument");
  if (body < 0 || body >= h->nbodies) return fail(PSM_ERR_ARG, "no body %d", body);
  if (h->recording) return fail(PSM_ERR_STATE, "two-way coupling while recording for psm_backward");
  if (h->remap_frozen) return fail(PSM_ERR_STATE, "two-way coupling with the remap frozen");
  if (h->slab) return fail(PSM_ERR_STATE, "two-way coupling of a z-slab (each slab sees part of the force)");
  const double* I = dyn->inertia;
  bool ok = dyn->mass > 0.0 && std::isfinite(dyn->mass);
  for (int k = 0; k < 9; ++k) ok = ok && std::isfinite(I[k]);
  for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(dyn->force_ext[k]) && std::isfinite(dyn->torque_ext[k]);
  // symmetric positive definite: symmetric, leading principal minors > 0
  ok = ok && I[1] == I[3] && I[2] == I[6] && I[5] == I[7];
  const double m2 = I[0] * I[4] - I[1] * I[3];
  const double det = I[0] * (I[4] * I[8] - I[5] * I[7]) - I[1] * (I[3] * I[8] - I[5] * I[6]) +
                     I[2] * (I[3] * I[7] - I[4] * I[6]);
  ok = ok && I[0] > 0.0 && m2 > 0.0 && det > 0.0;
  if (!ok) return fail(PSM_ERR_ARG, "body dynamics: mass must be > 0 and the inertia symmetric positive definite");
  if (!h->d_dyn) {
    PSM_CUDA(cudaMalloc(&h->d_dyn, sizeof(psm::BodyDyn) * PSM_MAX_BODIES), "body state allocation");
    PSM_CUDA(cudaMalloc(&h->d_dev_bodies, sizeof(DevBody) * PSM_MAX_BODIES), "body state allocation");
  }
  const HostBody& hb = h->body[body];
  psm::BodyDyn S;
  std::memset(&S, 0, sizeof S);
  body_pose(hb, h->step, S.Q, S.R);
  for (int k = 0; k < 3; ++k) {
    S.v[k] = hb.v[k];
    S.w[k] = hb.omega[k];
    S.Fext[k] = dyn->force_ext[k];
    S.Text[k] = dyn->torque_ext[k];
    S.lo[k] = hb.lo[k];
  }
  S.gx = (int)hb.gx;
  S.gy = (int)hb.gy;
  S.gz = (int)hb.gz;
  S.mass = dyn->mass;
  // inverse inertia by cofactors
  S.Ibinv[0] = (I[4] * I[8] - I[5] * I[7]) / det;
  S.Ibinv[1] = (I[2] * I[7] - I[1] * I[8]) / det;
  S.Ibinv[2] = (I[1] * I[5] - I[2] * I[4]) / det;
  S.Ibinv[3] = (I[5] * I[6] - I[3] * I[8]) / det;
  S.Ibinv[4] = (I[0] * I[8] - I[2] * I[6]) / det;
  S.Ibinv[5] = (I[2] * I[3] - I[0] * I[5]) / det;
  S.Ibinv[6] = (I[3] * I[7] - I[4] * I[6]) / det;
  S.Ibinv[7] = (I[1] * I[6] - I[0] * I[7]) / det;
  S.Ibinv[8] = (I[0] * I[4] - I[1] * I[3]) / det;
  // L = Q I Q^T omega
  double a[3], c[3];
  for (int i = 0; i < 3; ++i) a[i] = S.Q[i] * S.w[0] + S.Q[3 + i] * S.w[1] + S.Q[6 + i] * S.w[2];
  for (int i = 0; i < 3; ++i) c[i] = I[3 * i] * a[0] + I[3 * i + 1] * a[1] + I[3 * i + 2] * a[2];
  for (int i = 0; i < 3; ++i) S.L[i] = S.Q[3 * i] * c[0] + S.Q[3 * i + 1] * c[1] + S.Q[3 * i + 2] * c[2];
  const DevBody d = dev_body(h, body, h->step);  // this step's pose, as prescribed
  PSM_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  PSM_CUDA(cudaMemcpy(h->d_dyn + body, &S, sizeof S, cudaMemcpyHostToDevice), "body state upload");
  PSM_CUDA(cudaMemcpy(h->d_dev_bodies + body, &d, sizeof d, cudaMemcpyHostToDevice), "body state upload");
  h->free_mask |= 1u << body;
  return PSM_OK;
}

int psm_body_state(psm_handle h, int body, double* out) {
  if (!valid_handle(h) || !out) return fail(PSM_ERR_ARG, "psm_body_state: NULL argument");
  if (body < 0 || body >= h->nbodies) return fail(PSM_ERR_ARG, "no body %d", body);
  if ((h->free_mask >> body) & 1u) {
    psm::BodyDyn S;
    PSM_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
    PSM_CUDA(cudaMemcpy(&S, h->d_dyn + body, sizeof S, cudaMemcpyDeviceToHost), "body state read");
    for (int k = 0; k < 3; ++k) out[k] = S.R[k], out[3 + k] = S.v[k], out[15 + k] = S.w[k], out[18 + k] = S.L[k];
    for (int k = 0; k < 9; ++k) out[6 + k] = S.Q[k];
  } else {
    const HostBody& hb = h->body[body];
    double Q[9], R[3];
    body_pose(hb, h->remap_frozen ? h->frozen_step : h->step, Q, R);
    for (int k = 0; k < 3; ++k) out[k] = R[k], out[3 + k] = hb.v[k], out[15 + k] = hb.omega[k], out[18 + k] = 0.0;
    for (int k = 0; k < 9; ++k) out[6 + k] = Q[k];
  }
  return PSM_OK;
}

int psm_mass(psm_handle h, double* out) {
  if (!valid_handle(h) || !out) return fail(PSM_ERR_ARG, "psm_mass: NULL argument");
  IoParams p;
  io_base(h, p);
  p.z_begin = 0;
  p.z_end = (int)h->grid.nz;
  p.partials = h->d_partials;
  p.ticket = h->d_ticket;
  p.sum_out = h->d_sum;
  const long long cells = h->g.ncell;
  long long blocks = (cells + psm::PSM_THREADS - 1) / psm::PSM_THREADS;
  if (blocks > h->max_blocks) blocks = h->max_blocks;
  PSM_CUDA(psm::launch_mass(h->lat.storage, h->Q, p, (int)blocks, h->stream), "mass kernel");
  PSM_CUDA(cudaMemcpyAsync(out, h->d_sum, sizeof(double), cudaMemcpyDefault, h->stream), "mass download");
  PSM_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  {
    const int rc = check_err(h);
    if (rc != PSM_OK) return rc;
  }
  if (!std::isfinite(*out)) return fail(PSM_ERR_NONFINITE, "mass is NaN or Inf");
  return PSM_OK;
}

int psm_synchronize(psm_handle h) {
  if (!valid_handle(h)) return fail(PSM_ERR_ARG, "psm_synchronize: NULL handle");
  PSM_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  return check_err(h);
}

}  // extern "C"
