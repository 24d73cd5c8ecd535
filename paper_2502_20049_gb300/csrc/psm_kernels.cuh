// CUDA kernels of the PSM hot path (arXiv 2502.20049), templated on the PDF
// storage type, the stencil, the streaming access pattern and the fluid
// collision.  Included by one translation unit per storage precision.
//
//   k_step    one fused time step: load (AA / two-grid), remap of the geometry
//             field onto eps (Sec. 3), moments, B (Eq. 5/6), u_s = omega x r + v,
//             Omega^F (Eq. 2 / TRT), Omega^S (Eq. 7/8/9), PSM blend (Eq. 4),
//             streamed store (Eq. 1), force/torque (Eq. 10/11) reduced in FP64
//             with a deterministic order (per-warp, per-block, last-block sum).
//   k_import  write a natural state (or a uniform equilibrium) in a layout
//   k_export  read a state in its layout and write it natural, unshifted, FP64
//   k_macro   rho and u per cell (FP64)
//   k_mass    deterministic FP64 total mass
//   k_remap   eps per cell (remap only)
#pragma once

#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>

#include "psm_internal.h"

namespace psm {

// ---------------------------------------------------------------------------
// Lattice: D3Q27 velocities in the library's order; the first 19 are D3Q19.
// Pairs (2k-1, 2k) are opposite; 0 is the rest direction.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int lat_cx(int i) {
  constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
  return t[i];
}
__host__ __device__ __forceinline__ constexpr int lat_cy(int i) {
  constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1};
  return t[i];
}
__host__ __device__ __forceinline__ constexpr int lat_cz(int i) {
  constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ __forceinline__ constexpr int lat_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
template <int Q>
__host__ __device__ __forceinline__ constexpr double lat_w(int i) {
  // |c|^2 = 0, 1, 2, 3
  return Q == 19 ? (i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0))
                 : (i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0)));
}

// ---------------------------------------------------------------------------
// Storage conversions.  PDFs are stored shifted (f - w rho0).
// ---------------------------------------------------------------------------
template <class S>
struct Store;
template <>
struct Store<double> {
  using T = double;
  static __device__ __forceinline__ double ld(const double* p) { return *p; }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
  static __device__ __forceinline__ double from_double(double v) { return v; }
};
template <>
struct Store<float> {
  using T = float;
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
  static __device__ __forceinline__ float from_double(double v) { return (float)v; }
};
template <>
struct Store<__half> {
  using T = float;
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ __half from_double(double v) { return __double2half(v); }
};
template <>
struct Store<__nv_bfloat16> {
  using T = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ __nv_bfloat16 from_double(double v) { return __double2bfloat16(v); }
};

// Two 16-bit values of neighbouring cells (x even, x + 1) as one 32-bit word:
// the lower half is the cell at the lower address (16-bit storage types only).
template <class S>
struct Pair16 {
  template <class T>
  static __device__ __forceinline__ void unpack(unsigned, T& a, T& b) { a = b = T(0); }
  template <class T>
  static __device__ __forceinline__ unsigned pack(T, T) { return 0u; }
};
template <>
struct Pair16<__half> {
  static __device__ __forceinline__ void unpack(unsigned w, float& a, float& b) {
    __half2 h;
    memcpy(&h, &w, 4);
    a = __low2float(h);
    b = __high2float(h);
  }
  static __device__ __forceinline__ unsigned pack(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
  }
};
template <>
struct Pair16<__nv_bfloat16> {
  static __device__ __forceinline__ void unpack(unsigned w, float& a, float& b) {
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    a = __low2float(h);
    b = __high2float(h);
  }
  static __device__ __forceinline__ unsigned pack(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
  }
};

// ---------------------------------------------------------------------------
// Remap of one body onto one cell (Sec. 3).  The cell centre is taken into the
// body frame, X = Q_n^T (x_c - R_n); the 2^s sub-cells per axis whose block
// starts at the sub-grid point nearest to X - 1/2 are counted in the
// brick-packed field.  The start index a0_k = floor(r_k),
// r_k = ((X_k - 1/2) - lo_k) 2^s + 1/2, is the double evaluation of r_k with
// separately rounded operations in that order.  The kernel evaluates r_k in
// float from the exact-split affine form of remap_setup (high part exact, low
// part within rtol of the double value); a cell whose float r_k lies within
// rtol of an integer on some axis takes the double evaluation itself, so the
// decision always equals the double one (the fallback is rare: rtol is a few
// float round-offs, so about 6 rtol of the cells in a body's box take it).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long low_bits(int w) { return w >= 64 ? ~0ull : ((1ull << w) - 1ull); }

static __device__ __noinline__ int3 remap_start_double(const DevBody& b, int x, int y, int z) {
  const double n = (double)(1 << b.s);
  const double xc[3] = {(double)x + 0.5, (double)y + 0.5, (double)z + 0.5};
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = __dsub_rn(xc[k], b.R[k]);
  int a0[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double X = __dadd_rn(__dadd_rn(__dmul_rn(b.Qd[k], d[0]), __dmul_rn(b.Qd[3 + k], d[1])),
                               __dmul_rn(b.Qd[6 + k], d[2]));
    a0[k] = (int)floor(__dadd_rn(__dmul_rn(__dsub_rn(__dsub_rn(X, 0.5), b.lod[k]), n), 0.5));
  }
  return make_int3(a0[0], a0[1], a0[2]);
}

__device__ __forceinline__ float remap_eps(const DevBody& b, int x, int y, int z) {
  const int s = b.s;
  const int n = 1 << s;
  const float e0 = (float)(x - b.anchor[0]), e1 = (float)(y - b.anchor[1]), e2 = (float)(z - b.anchor[2]);
  int a0[3];
  bool near = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float hi = __fmaf_rn(b.Ghi[6 + k], e2, __fmaf_rn(b.Ghi[3 + k], e1, __fmaf_rn(b.Ghi[k], e0, b.Hhi[k])));
    const float lo = __fmaf_rn(b.Glo[6 + k], e2, __fmaf_rn(b.Glo[3 + k], e1, __fmaf_rn(b.Glo[k], e0, b.Hlo[k])));
    const float fh = floorf(hi);
    const float v = __fadd_rn(__fsub_rn(hi, fh), lo);  // hi - fh is exact
    const float fv = floorf(v);
    a0[k] = (int)fh + (int)fv;
    near = near || fminf(__fsub_rn(v, fv), __fsub_rn(__fadd_rn(fv, 1.0f), v)) <= b.rtol;
  }
  if (near) {
    const int3 a = remap_start_double(b, x, y, z);
    a0[0] = a.x;
    a0[1] = a.y;
    a0[2] = a.z;
  }
  // per axis up to two coarse cells: [o, n) of g and [0, o) of g + 1
  int gc[3], o[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gc[k] = a0[k] >> s;  // arithmetic shift = floor division
    o[k] = a0[k] & (n - 1);
  }
  const int dims[3] = {b.gx, b.gy, b.gz};
  // quick reject: the whole block lies outside the stored box
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int glast = gc[k] + (o[k] ? 1 : 0);
    if (glast < 0 || gc[k] >= dims[k]) return 0.0f;
  }
  // the block touches coarse cells {gc, gc + 1}^3 at most: none holds a set bit
  // where the occupancy byte is zero (then eps is exactly 0); the block bit of
  // 8^3 occupancy bytes is tested first (a small array that stays in L1,
  // where the bytes come from L2 or memory)
  if (b.occ8) {
    const long long bi = ((long long)((gc[2] + 1) >> 3) * b.o8y + ((gc[1] + 1) >> 3)) * b.o8x + ((gc[0] + 1) >> 3);
    if (!((__ldg(b.occ8 + (bi >> 5)) >> (unsigned)(bi & 31)) & 1u)) return 0.0f;
  }
  if (b.occ) {
    const long long oi = ((long long)(gc[2] + 1) * (b.gy + 1) + (gc[1] + 1)) * (long long)(b.gx + 1) + (gc[0] + 1);
    if (!__ldg(b.occ + oi)) return 0.0f;
  }
  int count = 0;
  const int nn = n * n;
  // s <= 2 (one word per brick, bit (z n + y) n + x): rowrep has bit r n set
  // for every row r < n^2, layrep bit l n^2 for every layer l < n
  const unsigned long long rowrep = s == 2 ? 0x1111111111111111ull : (s == 1 ? 0x55ull : 1ull);
  const unsigned long long layrep = s == 2 ? 0x0001000100010001ull : (s == 1 ? 0x11ull : 1ull);
  for (int sz = 0; sz < 2; ++sz) {
    if (sz == 1 && o[2] == 0) break;
    const int gz = gc[2] + sz;
    if (gz < 0 || gz >= b.gz) continue;
    const int za = sz ? 0 : o[2], zb = sz ? o[2] : n;
    for (int sy = 0; sy < 2; ++sy) {
      if (sy == 1 && o[1] == 0) break;
      const int gy = gc[1] + sy;
      if (gy < 0 || gy >= b.gy) continue;
      const int ya = sy ? 0 : o[1], yb = sy ? o[1] : n;
      for (int sx = 0; sx < 2; ++sx) {
        if (sx == 1 && o[0] == 0) break;
        const int gx = gc[0] + sx;
        if (gx < 0 || gx >= b.gx) continue;
        const int xa = sx ? 0 : o[0], xb = sx ? o[0] : n;
        const unsigned long long* brick =
            b.bricks + ((long long)((long long)gz * b.gy + gy) * b.gx + gx) * b.wpb;
        const unsigned long long xm = low_bits(xb - xa) << xa;
        if (s <= 2) {
          const unsigned long long ym = (low_bits(n * (yb - ya)) << (n * ya)) * layrep;
          const unsigned long long zm = low_bits(nn * (zb - za)) << (nn * za);
          const unsigned long long m = (xm * rowrep) & ym & zm;
          count += __popcll(__ldg(brick) & m);
        } else {
          // s = 3: word = z layer, bit y * 8 + x
          const unsigned long long m = (xm * 0x0101010101010101ull) & (low_bits(8 * (yb - ya)) << (8 * ya));
          for (int w = za; w < zb; ++w) count += __popcll(__ldg(brick + w) & m);
        }
      }
    }
  }
  return (float)count * (1.0f / (float)(n * nn));
}

// eps (min(1, sum over bodies)) and owner (argmax, lower id on ties; -1 if none)
__device__ __forceinline__ float cell_eps(const DevBody* bodies, int nb, int x, int y, int z, int& owner) {
  float sum = 0.0f, best = 0.0f;
  owner = -1;
  for (int bi = 0; bi < nb; ++bi) {
    const DevBody& b = bodies[bi];
    if (x >= b.x0 && x < b.x1 && y >= b.y0 && y < b.y1 && z >= b.z0 && z < b.z1) {
      const float e = remap_eps(b, x, y, z);
      sum += e;
      if (e > best) {
        best = e;
        owner = bi;
      }
    }
  }
  return fminf(sum, 1.0f);
}

// ---------------------------------------------------------------------------
// Neighbour offsets of a cell (periodic x, y; periodic or bounded z)
// ---------------------------------------------------------------------------
struct Nbr {
  // 32-bit unsigned offsets: cell indices are < 2^32 and the sum cell + off
  // wraps modulo 2^32 onto the neighbour's index
  unsigned dxm, dxp, dym, dyp, dzm, dzp;
  bool zlo_out, zhi_out;  // z - 1 (resp. z + 1) lies outside (ghost plane)
  __device__ __forceinline__ void init(const Grid3& g, int x, int y, int z) {
    const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
    dxm = (x == 0) ? nx - 1u : 0u - 1u;
    dxp = (x == g.nx - 1) ? 0u - (nx - 1u) : 1u;
    dym = (y == 0) ? (unsigned)(g.ny - 1) * nx : 0u - nx;
    dyp = (y == g.ny - 1) ? 0u - (unsigned)(g.ny - 1) * nx : nx;
    dzm = (z == 0) ? (unsigned)(g.nz - 1) * plane : 0u - plane;
    dzp = (z == g.nz - 1) ? 0u - (unsigned)(g.nz - 1) * plane : plane;
    const bool ghost = g.bc_z == PSM_BC_EQ_INLET_OUTLET;
    zlo_out = ghost && z == 0;
    zhi_out = ghost && z == g.nz - 1;
  }
  __device__ __forceinline__ unsigned off(int dx, int dy, int dz) const {
    return (dx < 0 ? dxm : (dx > 0 ? dxp : 0u)) + (dy < 0 ? dym : (dy > 0 ? dyp : 0u)) +
           (dz < 0 ? dzm : (dz > 0 ? dzp : 0u));
  }
  // x - c_i lies in a ghost plane: population i enters from the ghost plane
  __device__ __forceinline__ bool from_ghost(int cz) const { return (cz > 0 && zlo_out) || (cz < 0 && zhi_out); }
  // x + c_i lies in a ghost plane: population i leaves the domain
  __device__ __forceinline__ bool to_ghost(int cz) const { return (cz > 0 && zhi_out) || (cz < 0 && zlo_out); }
};

// s a for a lattice component s in {-1, 0, 1}, without multiplying (IEEE
// arithmetic keeps 0 * a, so products with the zero components are avoided)
template <class T>
__device__ __forceinline__ T csign(int c, T a) {
  return c > 0 ? a : (c < 0 ? -a : T(0));
}
// c_i . v over the non-zero components of c_i only
template <class T>
__device__ __forceinline__ T cdot(int i, T vx, T vy, T vz) {
  T r = T(0);
  bool h = false;
  if (lat_cx(i)) {
    r = csign(lat_cx(i), vx);
    h = true;
  }
  if (lat_cy(i)) {
    r = h ? r + csign(lat_cy(i), vy) : csign(lat_cy(i), vy);
    h = true;
  }
  if (lat_cz(i)) r = h ? r + csign(lat_cz(i), vz) : csign(lat_cz(i), vz);
  return r;
}

// Eq. 3 (sign-corrected) minus the storage shift w rho0, for velocity v:
//   f^eq_i(rho, v) - w_i rho0 = w_i (drho + rho (3 c.v + 4.5 (c.v)^2 - 1.5 v.v))
template <int Q, class T>
__device__ __forceinline__ T feq_shifted(int i, T drho, T rho, T vx, T vy, T vz, T vv) {
  const T cv = T(lat_cx(i)) * vx + T(lat_cy(i)) * vy + T(lat_cz(i)) * vz;
  return T(lat_w<Q>(i)) * (drho + rho * (T(3) * cv + T(4.5) * cv * cv - T(1.5) * vv));
}
// the same over the non-zero components of c_i only (fewer instructions; the
// adjoint kernel's form)
template <int Q, class T>
__device__ __forceinline__ T feq_shifted_nz(int i, T drho, T rho, T vx, T vy, T vz, T vv) {
  const T cv = cdot(i, vx, vy, vz);
  return T(lat_w<Q>(i)) * (drho + rho * (T(3) * cv + T(4.5) * cv * cv - T(1.5) * vv));
}

__device__ __forceinline__ int tile_coords(const Tiling& t, int tile, int& x, int& y, int& z) {
  const int tx = tile % t.ntx;
  const int r = tile / t.ntx;
  const int ty = r % t.nty;
  z = r / t.nty;
  x = tx * t.tx + (int)(threadIdx.x % t.tx);
  y = ty * t.ty + (int)(threadIdx.x / t.tx);
  return 0;
}

template <class V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Type of one cell's force/torque contribution and of its warp partial sum:
// the compute precision (FP64 arithmetic for FP64 storage; FP32 otherwise).
// The per-warp partials are added into FP64 block slots, and the block and
// grid sums are FP64 (on GB300 an FP64 instruction costs about 64 FP32 ones,
// so the 32-cell partials stay in the arithmetic's own precision).
template <class T>
using ft_t = typename std::conditional<sizeof(T) == 8, double, float>::type;

// Block-wide ordered reduction of per-block values v[0..ncomp) held in shared
// memory `blk` into partials[blockIdx.x]; the last block to finish sums all
// partials in a fixed order into out[0..ncomp).  Deterministic for a fixed grid.
__device__ __forceinline__ void grid_reduce(const double* blk, int ncomp, double* partials, unsigned int* ticket,
                                            double* out) {
  __shared__ unsigned int s_last;
  __shared__ double red[PSM_THREADS];
  if ((int)threadIdx.x < ncomp) {
    partials[(long long)blockIdx.x * ncomp + threadIdx.x] = blk[threadIdx.x];
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x) s += __ldcg(&partials[(long long)j * ncomp + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// ---------------------------------------------------------------------------
// The fused step kernel (persistent: blocks stride over row tiles).
// ---------------------------------------------------------------------------
// Resident blocks per SM the register allocation aims at (D3Q19 / D3Q27).
#ifndef PSM_MIN_BLOCKS_Q19
#define PSM_MIN_BLOCKS_Q19 3
#endif
#ifndef PSM_MIN_BLOCKS_Q27
#define PSM_MIN_BLOCKS_Q27 2
#endif
// Resident blocks per SM of a step kernel for storage S and stencil Q: FP64
// state needs twice the registers per PDF, so one block fewer (80 / 128 / 255
// registers per thread at 3 / 2 / 1 blocks of 256 threads).
// The cumulant operator (FL = 2, D3Q19) keeps about twice the values of
// BGK/TRT live: it aims at PSM_MIN_BLOCKS_CUM blocks (128 registers at 2),
// and FP64 at one.
#ifndef PSM_MIN_BLOCKS_CUM
#define PSM_MIN_BLOCKS_CUM 2
#endif
// The D3Q27 AA odd step in 2-byte storage (one cell per thread) fits 80
// registers without spills and runs three blocks, where its even step (two
// cells per thread) needs the 128-register budget of two.
template <class S, int Q, int FL = 0, int MODE = -1>
__host__ __device__ constexpr int step_min_blocks() {
  if (FL == 2) return sizeof(S) == 8 ? 1 : PSM_MIN_BLOCKS_CUM;
  if (Q == 27 && sizeof(S) == 2 && MODE == MODE_AA_ODD) return 3;
  return sizeof(S) == 8 ? (Q == 19 ? PSM_MIN_BLOCKS_Q19 - 1 : PSM_MIN_BLOCKS_Q27 - 1)
                        : (Q == 19 ? PSM_MIN_BLOCKS_Q19 : PSM_MIN_BLOCKS_Q27);
}

template <class T>
__device__ __forceinline__ const ConstT<T>& cst(const StepParams& p) {
  if constexpr (sizeof(T) == 4) return p.cf;
  else return p.cd;
}

// 1 / r: FP32 by rcp.approx refined with one Newton-Raphson step
// (a' = a + a (1 - r a)), within 1 ulp for the densities here (r near 1); FP64
// by IEEE division.
template <class T>
__device__ __forceinline__ T recip(T r) {
  if constexpr (sizeof(T) == 4) {
    float a;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(r));
    return fmaf(a, fmaf(-r, a, 1.0f), a);
  } else {
    return T(1) / r;
  }
}

// |c_i|^2: the weight class of direction i (0 rest, 1 axis, 2 face diagonal, 3 corner)
__host__ __device__ __forceinline__ constexpr int lat_cls(int i) {
  return lat_cx(i) * lat_cx(i) + lat_cy(i) * lat_cy(i) + lat_cz(i) * lat_cz(i);
}

// Separately rounded operations (never contracted or reordered by the
// compiler): the fluid collision computes the same bits in every kernel that
// inlines it.
template <class T>
__device__ __forceinline__ T r_add(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fadd_rn(a, b);
  else return __dadd_rn(a, b);
}
template <class T>
__device__ __forceinline__ T r_sub(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fsub_rn(a, b);
  else return __dsub_rn(a, b);
}
template <class T>
__device__ __forceinline__ T r_mul(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fmul_rn(a, b);
  else return __dmul_rn(a, b);
}
template <class T>
__device__ __forceinline__ T r_fma(T a, T b, T c) {
  if constexpr (sizeof(T) == 4) return __fmaf_rn(a, b, c);
  else return __fma_rn(a, b, c);
}
// a + s b for a lattice component s = +-1
template <class T>
__device__ __forceinline__ T r_addc(T a, int s, T b) {
  return s > 0 ? r_add(a, b) : r_sub(a, b);
}
template <class T>
__device__ __forceinline__ T r_div(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fdiv_rn(a, b);
  else return __ddiv_rn(a, b);
}

// Density deviation, density and velocity of one cell from its shifted PDFs,
// summed over opposite pairs (i, i + 1): drho = f_0 + sum (f_i + f_i+1),
// j = sum c_i (f_i - f_i+1).
template <class T, int Q>
__device__ __forceinline__ void moments(const T (&f)[Q], T rho0, T& drho, T& rho, T& ux, T& uy, T& uz, T& uu) {
  T d = f[0], jx = T(0), jy = T(0), jz = T(0);
  bool hx = false, hy = false, hz = false;  // compile-time after unrolling
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const T sp = r_add(f[i], f[i + 1]), dm = r_sub(f[i], f[i + 1]);
    d = r_add(d, sp);
    if (lat_cx(i)) {
      jx = hx ? r_addc(jx, lat_cx(i), dm) : (lat_cx(i) > 0 ? dm : -dm);
      hx = true;
    }
    if (lat_cy(i)) {
      jy = hy ? r_addc(jy, lat_cy(i), dm) : (lat_cy(i) > 0 ? dm : -dm);
      hy = true;
    }
    if (lat_cz(i)) {
      jz = hz ? r_addc(jz, lat_cz(i), dm) : (lat_cz(i) > 0 ? dm : -dm);
      hz = true;
    }
  }
  drho = d;
  rho = r_add(rho0, d);
  const T inv_rho = recip(rho);
  ux = r_mul(jx, inv_rho);
  uy = r_mul(jy, inv_rho);
  uz = r_mul(jz, inv_rho);
  uu = r_fma(uz, uz, r_fma(uy, uy, r_mul(ux, ux)));
}

// c_i . u with separately rounded operations
template <class T>
__device__ __forceinline__ T c_dot(int i, T ux, T uy, T uz) {
  T cu = T(0);
  bool h = false;
  if (lat_cx(i)) {
    cu = lat_cx(i) > 0 ? ux : -ux;
    h = true;
  }
  if (lat_cy(i)) {
    cu = h ? r_addc(cu, lat_cy(i), uy) : (lat_cy(i) > 0 ? uy : -uy);
    h = true;
  }
  if (lat_cz(i)) cu = h ? r_addc(cu, lat_cz(i), uz) : (lat_cz(i) > 0 ? uz : -uz);
  return cu;
}

// feq_shifted with separately rounded operations (the PSM cells of the
// cumulant step): w_i (drho + rho (3 c.v + 4.5 (c.v)^2 - 1.5 v.v))
template <int Q, class T>
__device__ __forceinline__ T feq_shifted_r(int i, T drho, T rho, T vx, T vy, T vz, T vv) {
  const T cv = c_dot(i, vx, vy, vz);
  const T q = r_fma(r_mul(T(4.5), cv), cv, r_fma(T(3), cv, r_mul(T(-1.5), vv)));
  return r_mul(T(lat_w<Q>(i)), r_fma(rho, q, drho));
}

// Pure fluid cell: f* = f + Omega^F (TRT; BGK is the case omega+ = omega- =
// 1/tau).  Per opposite pair (i, j), c_j = -c_i, with s = f_i + f_j and
// d = f_i - f_j the shifted equilibrium splits into
//   even = w (drho + rho (4.5 (c.u)^2 - 1.5 u.u)),  odd = 3 w rho (c.u),
//   f^eq_i - w rho0 = even + odd,  f^eq_j - w rho0 = even - odd,
// and the relaxed pair is f*_i = p + m, f*_j = p - m with
//   p = (1 - omega+) s / 2 + omega+ even,  m = (1 - omega-) d / 2 + omega- odd.
// The products of omega+-, the weight and the numeric factors are host
// constants per weight class (ConstT pw, pk, pd); f_i and f_j are not needed
// once s and d are formed.
template <class T, bool UNIT>
__device__ __forceinline__ void cumulant_relax(const ConstT<T>& C, T (&f)[19], T drho, T rho, T ux, T uy, T uz);

template <class T, int Q, int FL>
__device__ __forceinline__ void fluid_relax(const ConstT<T>& C, T (&f)[Q], T drho, T rho, T ux, T uy, T uz, T uu) {
  if constexpr (FL == 2) {
    static_assert(Q == 19, "the cumulant operator is defined for D3Q19");
    if (C.cum_unit) cumulant_relax<T, true>(C, f, drho, rho, ux, uy, uz);
    else cumulant_relax<T, false>(C, f, drho, rho, ux, uy, uz);
    return;
  }
  const T base = r_fma(T(-1.5), r_mul(rho, uu), drho);
  constexpr int NC = Q == 27 ? 4 : 3;
  T A[NC], K[NC], D[NC];  // per class: omega+ w base, 4.5 omega+ w rho, 3 omega- w rho
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    A[c] = r_mul(C.pw[c], base);
    K[c] = r_mul(C.pk[c], rho);
    D[c] = r_mul(C.pd[c], rho);
  }
  f[0] = r_fma(C.omp1, f[0], A[0]);
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int j = i + 1, c = lat_cls(i);
    const T cu = c_dot(i, ux, uy, uz);
    const T sp = r_add(f[i], f[j]), dm = r_sub(f[i], f[j]);
    const T pe = r_fma(C.hp1, sp, r_fma(K[c], r_mul(cu, cu), A[c]));
    const T mo = r_fma(C.hm1, dm, r_mul(D[c], cu));
    f[i] = r_add(pe, mo);
    f[j] = r_sub(pe, mo);
  }
}

// Cumulant collision of one D3Q19 cell (Geier et al. 2015: listed in Sec. 2.2,
// the operator of every performance run in Sec. 5.1), restricted to the 19
// moments D3Q19 resolves, from the shifted PDFs f (f - w rho0), in place.
//   raw moments of the shifted PDFs, plane by plane (D3Q19 has no corner
//     directions, so the x-y face diagonals alone carry c_x^2 c_y^2, c_x^2 c_y,
//     c_x c_y^2 and c_x c_y);
//   central moments k_abc about u, kept as deviations from the fluid at rest
//     (k^_200 = k_200 - rho/3, k^_220 = k_220 - rho/9): every term is then of
//     the size of u^2 or the non-equilibrium part, so FP32 loses nothing to
//     cancellation against rho/3 or rho/9;
//   relaxation: off-diagonal and deviatoric second order with 1 - 1/tau, the
//     trace with 1 - omega_bulk, third order with 1 - omega_3, the fourth-order
//     cumulants C_220 = k_220 - (k_200 k_020 + 2 k_110^2) / rho with
//     1 - omega_4 (host constants cum1[0..3]); with the default rates (bulk,
//     third and fourth order 1, UNIT) the trace, third- and fourth-order
//     cumulants are set to equilibrium without computing them;
//   raw moments of the result by the inverse shift, then the D3Q19 PDFs in
//     closed form: f(sx, sy, 0) = (m_220 + sx m_120 + sy m_210 + sx sy m_110) / 4,
//     f(s, 0, 0) = ((m_200 - m_220 - m_202) + s (m_100 - m_120 - m_102)) / 2,
//     f_0 = m_000 - m_200 - m_020 - m_002 + m_220 + m_202 + m_022.
// Operations are separately rounded (same bits in every kernel that inlines it).
template <class T, bool UNIT>
__device__ __forceinline__ void cumulant_relax(const ConstT<T>& C, T (&f)[19], T drho, T rho, T ux, T uy, T uz) {
  auto ad = [](T a, T b) { return r_add(a, b); };
  auto sb = [](T a, T b) { return r_sub(a, b); };
  auto ml = [](T a, T b) { return r_mul(a, b); };
  auto fm = [](T a, T b, T c) { return r_fma(a, b, c); };
  const T third = T(1.0 / 3.0), ninth = T(1.0 / 9.0);
  // ---- raw moments of the shifted PDFs ----
  const T Ax = ad(f[1], f[2]), Bx = sb(f[1], f[2]);
  const T Ay = ad(f[3], f[4]), By = sb(f[3], f[4]);
  const T Az = ad(f[5], f[6]), Bz = sb(f[5], f[6]);
  T Sxy, Mxy, Xxy, Yxy, Sxz, Mxz, Xxz, Zxz, Syz, Myz, Yyz, Zyz;
  {
    // group (a, b) with f[k] = (+,+), f[k+1] = (-,-), f[k+2] = (+,-), f[k+3] = (-,+)
    auto group = [&](int k, T& S, T& M, T& A, T& B) {
      const T p1 = ad(f[k], f[k + 1]), m1 = sb(f[k], f[k + 1]);
      const T p2 = ad(f[k + 2], f[k + 3]), m2 = sb(f[k + 2], f[k + 3]);
      S = ad(p1, p2);  // sum c_a^2 c_b^2 f
      M = sb(p1, p2);  // sum c_a c_b f
      A = ad(m1, m2);  // sum c_a f (= sum c_a c_b^2 f)
      B = sb(m1, m2);  // sum c_b f (= sum c_a^2 c_b f)
    };
    group(7, Sxy, Mxy, Xxy, Yxy);
    group(11, Sxz, Mxz, Xxz, Zxz);
    group(15, Syz, Myz, Yyz, Zyz);
  }
  const T jx = ad(ad(Bx, Xxy), Xxz), jy = ad(ad(By, Yxy), Yyz), jz = ad(ad(Bz, Zxz), Zyz);
  const T m200 = ad(ad(Ax, Sxy), Sxz), m020 = ad(ad(Ay, Sxy), Syz), m002 = ad(ad(Az, Sxz), Syz);
  // ---- central moments (deviation form) ----
  const T dt = ml(drho, third), dn = ml(drho, ninth);
  const T rux = ml(rho, ux), ruy = ml(rho, uy), ruz = ml(rho, uz);
  const T k200 = sb(m200, fm(rux, ux, dt)), k020 = sb(m020, fm(ruy, uy, dt)), k002 = sb(m002, fm(ruz, uz, dt));
  const T k110 = sb(Mxy, ml(rux, uy)), k101 = sb(Mxz, ml(rux, uz)), k011 = sb(Myz, ml(ruy, uz));
  const T uxx = ml(ux, ux), uyy = ml(uy, uy), uzz = ml(uz, uz);
  const T s1 = C.cum1[0];
  const T inv_rho = recip(rho);
  const T p110 = ml(s1, k110), p101 = ml(s1, k101), p011 = ml(s1, k011);
  const T d1 = ml(s1, sb(k200, k020)), d2 = ml(s1, sb(k200, k002));
  // relaxed second-order (deviatoric with 1 - 1/tau, trace with 1 - omega_bulk),
  // third-order (k_aab) and fourth-order (k^_aabb) central moments
  T p200, p020, p002, p210 = T(0), p120 = T(0), p201 = T(0), p102 = T(0), p021 = T(0), p012 = T(0);
  T p220, p202, p022;
  // k^_aabb of a Gaussian-like closure: (p_aa + p_bb)/3 + (p_aa p_bb + 2 p_ab^2)/rho
  auto closure = [&](T paa, T pbb, T pab) {
    return fm(third, ad(paa, pbb), ml(fm(paa, pbb, ml(ml(T(2), pab), pab)), inv_rho));
  };
  if constexpr (UNIT) {
    // bulk, third- and fourth-order rates 1: trace, third-order and fourth-order
    // cumulants take their equilibrium values (0 in deviation form)
    p200 = ml(ad(d1, d2), third);
    p020 = ml(fm(T(-2), d1, d2), third);
    p002 = ml(fm(T(-2), d2, d1), third);
    p220 = closure(p200, p020, p110);
    p202 = closure(p200, p002, p101);
    p022 = closure(p020, p002, p011);
  } else {
    const T b1 = C.cum1[1], t1 = C.cum1[2], q1 = C.cum1[3];
    const T r0t = ml(C.rho0, third);
    const T M200 = ad(m200, r0t), M020 = ad(m020, r0t), M002 = ad(m002, r0t);  // full raw c_a^2 moments
    const T n2ux = ml(T(-2), ux), n2uy = ml(T(-2), uy), n2uz = ml(T(-2), uz);
    // k_aab = m_aab - u_b M_aa - 2 u_a k_ab
    const T k210 = fm(n2ux, k110, fm(-uy, M200, Yxy)), k120 = fm(n2uy, k110, fm(-ux, M020, Xxy));
    const T k201 = fm(n2ux, k101, fm(-uz, M200, Zxz)), k102 = fm(n2uz, k101, fm(-ux, M002, Xxz));
    const T k021 = fm(n2uy, k011, fm(-uz, M020, Zyz)), k012 = fm(n2uz, k011, fm(-uy, M002, Yyz));
    // k^_aabb = (m_aabb - drho/9) - 2 u_b k_aab - 2 u_a k_abb - 4 u_a u_b k_ab - u_b^2 k^_aa
    //           - u_a^2 k^_bb - rho (u_a^2 + u_b^2) / 3 - rho u_a^2 u_b^2
    auto k4 = [&](T S, T kaab, T kabb, T ua, T ub, T uaa, T ubb, T kab, T kaa, T kbb) {
      T r = sb(S, dn);
      r = fm(ml(T(-2), ub), kaab, r);
      r = fm(ml(T(-2), ua), kabb, r);
      r = fm(ml(T(-4), ml(ua, ub)), kab, r);
      r = fm(-ubb, kaa, r);
      r = fm(-uaa, kbb, r);
      r = fm(-ml(rho, third), ad(uaa, ubb), r);
      return fm(-ml(rho, uaa), ubb, r);
    };
    const T k220 = k4(Sxy, k210, k120, ux, uy, uxx, uyy, k110, k200, k020);
    const T k202 = k4(Sxz, k201, k102, ux, uz, uxx, uzz, k101, k200, k002);
    const T k022 = k4(Syz, k021, k012, uy, uz, uyy, uzz, k011, k020, k002);
    const T tr = ml(b1, ad(ad(k200, k020), k002));
    p200 = ml(ad(ad(tr, d1), d2), third);
    p020 = ml(ad(fm(T(-2), d1, tr), d2), third);
    p002 = ml(fm(T(-2), d2, ad(tr, d1)), third);
    p210 = ml(t1, k210), p120 = ml(t1, k120), p201 = ml(t1, k201);
    p102 = ml(t1, k102), p021 = ml(t1, k021), p012 = ml(t1, k012);
    // fourth order: C = k^_aabb - closure(k), relaxed with 1 - omega_4, plus closure(p)
    auto c4 = [&](T k, T kaa, T kbb, T kab) {
      return sb(fm(-third, ad(kaa, kbb), k), ml(fm(kaa, kbb, ml(ml(T(2), kab), kab)), inv_rho));
    };
    p220 = fm(q1, c4(k220, k200, k020, k110), closure(p200, p020, p110));
    p202 = fm(q1, c4(k202, k200, k002, k101), closure(p200, p002, p101));
    p022 = fm(q1, c4(k022, k020, k002, k011), closure(p020, p002, p011));
  }
  // ---- raw moments of the result (shifted PDFs) ----
  const T n200 = fm(rux, ux, ad(p200, dt)), n020 = fm(ruy, uy, ad(p020, dt)), n002 = fm(ruz, uz, ad(p002, dt));
  const T n110 = fm(rux, uy, p110), n101 = fm(rux, uz, p101), n011 = fm(ruy, uz, p011);
  const T rt = ml(rho, third);
  const T F200 = fm(rux, ux, ad(p200, rt)), F020 = fm(ruy, uy, ad(p020, rt)), F002 = fm(ruz, uz, ad(p002, rt));
  const T n2 = T(2);
  // m_aab = k_aab + u_b F_aa + 2 u_a k_ab
  auto b3 = [&](T paab, T ub, T Faa, T ua, T pab) {
    if constexpr (UNIT) return fm(ml(n2, ua), pab, ml(ub, Faa));
    else return fm(ml(n2, ua), pab, fm(ub, Faa, paab));
  };
  const T n210 = b3(p210, uy, F200, ux, p110), n120 = b3(p120, ux, F020, uy, p110);
  const T n201 = b3(p201, uz, F200, ux, p101), n102 = b3(p102, ux, F002, uz, p101);
  const T n021 = b3(p021, uz, F020, uy, p011), n012 = b3(p012, uy, F002, uz, p011);
  // m_aabb = k^_aabb + drho/9 + 2 u_b k_aab + 2 u_a k_abb + 4 u_a u_b k_ab + u_b^2 (k^_aa + rho/3)
  //          + u_a^2 (k^_bb + rho/3) + rho u_a^2 u_b^2
  auto b4 = [&](T k, T kaab, T kabb, T ua, T ub, T uaa, T ubb, T kab, T kaa, T kbb) {
    T r = ad(k, dn);
    if constexpr (!UNIT) {
      r = fm(ml(n2, ub), kaab, r);
      r = fm(ml(n2, ua), kabb, r);
    }
    r = fm(ml(T(4), ml(ua, ub)), kab, r);
    r = fm(ubb, ad(kaa, rt), r);
    r = fm(uaa, ad(kbb, rt), r);
    return fm(ml(rho, uaa), ubb, r);
  };
  const T n220 = b4(p220, p210, p120, ux, uy, uxx, uyy, p110, p200, p020);
  const T n202 = b4(p202, p201, p102, ux, uz, uxx, uzz, p101, p200, p002);
  const T n022 = b4(p022, p021, p012, uy, uz, uyy, uzz, p011, p020, p002);
  // ---- PDFs ----
  const T qtr = T(0.25), hf = T(0.5);
  auto ungroup = [&](int k, T S, T M, T A, T B) {
    const T a = ad(S, M), b = sb(S, M), p = ad(A, B), q = sb(A, B);
    f[k] = ml(qtr, ad(a, p));
    f[k + 1] = ml(qtr, sb(a, p));
    f[k + 2] = ml(qtr, ad(b, q));
    f[k + 3] = ml(qtr, sb(b, q));
  };
  ungroup(7, n220, n110, n120, n210);
  ungroup(11, n202, n101, n102, n201);
  ungroup(15, n022, n011, n012, n021);
  auto axis = [&](int k, T e, T o) {
    f[k] = ml(hf, ad(e, o));
    f[k + 1] = ml(hf, sb(e, o));
  };
  axis(1, sb(sb(n200, n220), n202), sb(sb(jx, n120), n102));
  axis(3, sb(sb(n020, n220), n022), sb(sb(jy, n210), n012));
  axis(5, sb(sb(n002, n202), n022), sb(sb(jz, n201), n021));
  f[0] = ad(ad(ad(sb(sb(sb(drho, n200), n020), n002), n220), n202), n022);
}

// One cell's PSM update in registers, from its pre-collision (shifted) PDFs f:
// remap (Sec. 3), B (Eq. 5/6), moments, u_s = omega x r + v, Omega^F (Eq. 2 /
// TRT), Omega^S (Eq. 7/8/9), blend (Eq. 4).  f becomes the post-collision
// state.  For a cell in contact with a body (B > 0) ft receives the force and
// torque on the body (minus Eq. 10 / 11 per cell, about R_n).  A cell with
// B = 0 takes exactly the arithmetic of fluid_relax.
template <class T, int Q, int FL>
__device__ __forceinline__ void psm_collide(const StepParams& p, const DevBody* bodies, T (&f)[Q], int x, int y,
                                            int z, unsigned cell, int& owner, bool& solid_cell, ft_t<T> (&ft)[6]) {
  // (x, y, z): world cell indices (z includes the slab offset); cell: this grid's index
  const ConstT<T>& C = cst<T>(p);
  const T om_a = C.om_a, om_b = C.om_b;
  const T inv_tau = C.inv_tau;
  // ---- remap (Sec. 3) and weighting (Eq. 5/6) ----
  // Every operation below is separately rounded (r_*): a PSM cell gets the
  // same bits in every kernel and loop shape that inlines this function.
  const float epsf = cell_eps(bodies, p.nbodies, x, y, z, owner);
  T eps = T(epsf);
  if (p.delta) eps = r_add(eps, T(p.delta[cell]));
  T Bw = eps;
  if (p.weighting == PSM_B_TAU_WEIGHTED && eps != T(0)) {  // eps = 0 gives B = eps exactly
    const T t = C.tmh;
    Bw = r_div(r_mul(eps, t), r_add(r_sub(T(1), eps), t));
  }
  T drho, rho, ux, uy, uz, uu;
  moments<T, Q>(f, C.rho0, drho, rho, ux, uy, uz, uu);
  solid_cell = Bw != T(0);
  if (!solid_cell) {
    fluid_relax<T, Q, FL>(C, f, drho, rho, ux, uy, uz, uu);
    return;
  }
  // ---- PSM cell: f* = f + (1 - B) Omega^F + B Omega^S (Eq. 4) ----
  T usx = 0, usy = 0, usz = 0;
  T rx = 0, ry = 0, rz = 0;  // lever arm x_c - R (Eq. 11)
  if (owner >= 0) {
    const DevBody& b = bodies[owner];
    T wx, wy, wz, vx, vy, vz;
    if constexpr (sizeof(T) == 4) {
      rx = r_sub(r_add(T(x), T(0.5)), b.Rf[0]);
      ry = r_sub(r_add(T(y), T(0.5)), b.Rf[1]);
      rz = r_sub(r_add(T(z), T(0.5)), b.Rf[2]);
      wx = b.omegaf[0], wy = b.omegaf[1], wz = b.omegaf[2];
      vx = b.vf[0], vy = b.vf[1], vz = b.vf[2];
    } else {
      rx = r_sub(r_add((double)x, 0.5), b.R[0]);
      ry = r_sub(r_add((double)y, 0.5), b.R[1]);
      rz = r_sub(r_add((double)z, 0.5), b.R[2]);
      wx = b.omega[0], wy = b.omega[1], wz = b.omega[2];
      vx = b.v[0], vy = b.v[1], vz = b.v[2];
    }
    // u_s = omega x r + v (Eq. 7-9)
    usx = r_add(r_sub(r_mul(wy, rz), r_mul(wz, ry)), vx);
    usy = r_add(r_sub(r_mul(wz, rx), r_mul(wx, rz)), vy);
    usz = r_add(r_sub(r_mul(wx, ry), r_mul(wy, rx)), vz);
  }
  const T usus = r_fma(usz, usz, r_fma(usy, usy, r_mul(usx, usx)));
  const T omB = r_sub(T(1), Bw);
  // cumulant: Omega^F = C(f) - f from the relaxed copy fc
  T fc[Q];
  if constexpr (FL == 2) {
#pragma unroll
    for (int i = 0; i < Q; ++i) fc[i] = f[i];
    fluid_relax<T, Q, FL>(C, fc, drho, rho, ux, uy, uz, uu);
  }
  T gx = 0, gy = 0, gz = 0;  // sum_i Omega^S_i c_i
  if constexpr (FL == 2) {
    {
      const T n0 = r_sub(f[0], feq_shifted_r<Q, T>(0, drho, rho, ux, uy, uz, uu));
      const T m0 = r_sub(f[0], feq_shifted_r<Q, T>(0, drho, rho, usx, usy, usz, usus));
      const T of = r_sub(fc[0], f[0]);
      T os;
      if (p.solid == PSM_SC1) os = r_sub(n0, m0);
      else if (p.solid == PSM_SC2) os = r_mul(-m0, inv_tau);
      else os = T(0);
      f[0] = r_fma(Bw, os, r_fma(omB, of, f[0]));
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int j = i + 1;
      const T ni = r_sub(f[i], feq_shifted_r<Q, T>(i, drho, rho, ux, uy, uz, uu));
      const T nj = r_sub(f[j], feq_shifted_r<Q, T>(j, drho, rho, ux, uy, uz, uu));
      const T mi = r_sub(f[i], feq_shifted_r<Q, T>(i, drho, rho, usx, usy, usz, usus));
      const T mj = r_sub(f[j], feq_shifted_r<Q, T>(j, drho, rho, usx, usy, usz, usus));
      const T ofi = r_sub(fc[i], f[i]), ofj = r_sub(fc[j], f[j]);
      T osi, osj;
      if (p.solid == PSM_SC1) {
        osi = r_sub(nj, mi);
        osj = r_sub(ni, mj);
      } else if (p.solid == PSM_SC2) {
        osi = r_mul(-mi, inv_tau);
        osj = r_mul(-mj, inv_tau);
      } else {
        osi = r_sub(mj, mi);
        osj = r_sub(mi, mj);
      }
      f[i] = r_fma(Bw, osi, r_fma(omB, ofi, f[i]));
      f[j] = r_fma(Bw, osj, r_fma(omB, ofj, f[j]));
      // c_j = -c_i: sum_i Omega^S_i c_i over the pair
      const T d = r_sub(osi, osj);
      if (lat_cx(i)) gx = r_addc(gx, lat_cx(i), d);
      if (lat_cy(i)) gy = r_addc(gy, lat_cy(i), d);
      if (lat_cz(i)) gz = r_addc(gz, lat_cz(i), d);
    }
  } else {
    // BGK / TRT in pair form (c_j = -c_i).  With s = f_i + f_j, d = f_i - f_j
    // and the equilibria split into even and odd parts, f^eq_i,j - w rho0 =
    // ev +- od at u and evs +- ods at u_s, the half sums and differences
    //   n+ = s/2 - ev, n- = d/2 - od,  m+ = s/2 - evs, m- = d/2 - ods
    // give Omega^F_i,j = -omega+ n+ -+ omega- n- and
    //   SC1: Omega^S_i,j = n_j - m_i, n_i - m_j = (n+ - m+) +- (-n- - m-),
    //   SC2: -(m+ +- m-) / tau,   SC3: m_j - m_i, m_i - m_j = +-(-2 m-);
    // then f*_i,j = P +- M with P = s/2 + (1 - B) OmF+ + B OmS+ and
    // M = d/2 + (1 - B) OmF- + B OmS-, and the pair adds 2 OmS- c_i to
    // sum_i Omega^S_i c_i.
    const T wp = r_add(om_a, om_b), wm = r_sub(om_a, om_b);
    const T bu = r_fma(T(-1.5), r_mul(rho, uu), drho), bs = r_fma(T(-1.5), r_mul(rho, usus), drho);
    {
      const T w0 = T(lat_w<Q>(0));
      const T n0 = r_fma(-w0, bu, f[0]), m0 = r_fma(-w0, bs, f[0]);
      T os;
      if (p.solid == PSM_SC1) os = r_sub(n0, m0);
      else if (p.solid == PSM_SC2) os = r_mul(-m0, inv_tau);
      else os = T(0);
      f[0] = r_fma(Bw, os, r_fma(omB, r_mul(-wp, n0), f[0]));
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int j = i + 1;
      const T w = T(lat_w<Q>(i));
      const T wr = r_mul(w, rho);
      const T cu = c_dot(i, ux, uy, uz), cs = c_dot(i, usx, usy, usz);
      const T k45 = r_mul(T(4.5), wr), k3 = r_mul(T(3), wr);
      const T ev = r_fma(k45, r_mul(cu, cu), r_mul(w, bu)), od = r_mul(k3, cu);
      const T evs = r_fma(k45, r_mul(cs, cs), r_mul(w, bs)), ods = r_mul(k3, cs);
      const T hs = r_mul(T(0.5), r_add(f[i], f[j])), hd = r_mul(T(0.5), r_sub(f[i], f[j]));
      const T np = r_sub(hs, ev), nm = r_sub(hd, od), mp = r_sub(hs, evs), mm = r_sub(hd, ods);
      T sp, sm;
      if (p.solid == PSM_SC1) {
        sp = r_sub(np, mp);
        sm = r_sub(-nm, mm);
      } else if (p.solid == PSM_SC2) {
        sp = r_mul(-mp, inv_tau);
        sm = r_mul(-mm, inv_tau);
      } else {
        sp = T(0);
        sm = r_mul(T(-2), mm);
      }
      const T P = r_fma(Bw, sp, r_fma(omB, r_mul(-wp, np), hs));
      const T M = r_fma(Bw, sm, r_fma(omB, r_mul(-wm, nm), hd));
      f[i] = r_add(P, M);
      f[j] = r_sub(P, M);
      const T d = r_mul(T(2), sm);
      if (lat_cx(i)) gx = r_addc(gx, lat_cx(i), d);
      if (lat_cy(i)) gy = r_addc(gy, lat_cy(i), d);
      if (lat_cz(i)) gz = r_addc(gz, lat_cz(i), d);
    }
  }
  if (owner >= 0) {
    // Eq. 10 / 11 per cell, in the arithmetic's precision (ft_t); the body
    // receives minus the solid's momentum transfer
    const T Gx = r_mul(Bw, gx), Gy = r_mul(Bw, gy), Gz = r_mul(Bw, gz);
    ft[0] = -Gx;
    ft[1] = -Gy;
    ft[2] = -Gz;
    ft[3] = -r_sub(r_mul(ry, Gz), r_mul(rz, Gy));
    ft[4] = -r_sub(r_mul(rz, Gx), r_mul(rx, Gz));
    ft[5] = -r_sub(r_mul(rx, Gy), r_mul(ry, Gx));
  }
}

// Streaming indices of one cell: the index of x + c for c in {-1, 0, 1}^3 is
// zc[cz + 1] + dy[cy + 1] + dx[cx + 1] (mod 2^32; cell indices are < 2^32),
// periodic in x and y, and in z (where z ends in ghost planes the callers
// drop the populations that cross them).
struct Stencil {
  unsigned zc[3], dy[3], dx[3];
  __device__ __forceinline__ void init(const Grid3& g, int x, int y, int z, unsigned cell) {
    const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
    dx[0] = (x == 0) ? nx - 1u : 0u - 1u;
    dx[1] = 0u;
    dx[2] = (x == g.nx - 1) ? 0u - (nx - 1u) : 1u;
    dy[0] = (y == 0) ? (unsigned)(g.ny - 1) * nx : 0u - nx;
    dy[1] = 0u;
    dy[2] = (y == g.ny - 1) ? 0u - (unsigned)(g.ny - 1) * nx : nx;
    zc[0] = cell + ((z == 0) ? (unsigned)(g.nz - 1) * plane : 0u - plane);
    zc[1] = cell;
    zc[2] = cell + ((z == g.nz - 1) ? 0u - (unsigned)(g.nz - 1) * plane : plane);
  }
  __device__ __forceinline__ unsigned at(int cx, int cy, int cz) const { return zc[cz + 1] + dy[cy + 1] + dx[cx + 1]; }
};

// Position of a z plane against the ghost planes (never set for periodic z).
struct ZGhost {
  bool lo, hi;  // z - 1 (resp. z + 1) lies in a ghost plane
  __device__ __forceinline__ void init(const Grid3& g, int z) {
    const bool ghost = g.bc_z == PSM_BC_EQ_INLET_OUTLET;
    lo = ghost && z == 0;
    hi = ghost && z == g.nz - 1;
  }
  // x - c_i lies in a ghost plane: population i enters from it
  __device__ __forceinline__ bool from(int cz) const { return (cz > 0 && lo) || (cz < 0 && hi); }
  // x + c_i lies in a ghost plane: population i leaves the domain
  __device__ __forceinline__ bool to(int cz) const { return (cz > 0 && hi) || (cz < 0 && lo); }
};

// Streamed store (Eq. 1) of one cell's post-collision PDFs:
//   AA even  own cell, slot opp(i);
//   AA odd   cell x + c_i, slot i;
//   TG       cell x + c_i, slot i of the other buffer;
// with GHOST, populations that leave the domain through a ghost plane are dropped.
template <class S, int Q, int MODE, bool GHOST, class T>
__device__ __forceinline__ void psm_store(const StepParams& p, const Stencil& sn, const ZGhost& zg, unsigned cell,
                                          const T (&f)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (MODE == MODE_AA_EVEN) {
      Store<S>::st(static_cast<S*>(p.dst_slot[lat_opp(i)]) + cell, f[i]);
    } else if (!GHOST || !zg.to(lat_cz(i))) {
      Store<S>::st(static_cast<S*>(p.dst_slot[i]) + sn.at(lat_cx(i), lat_cy(i), lat_cz(i)), f[i]);
    }
  }
}

// Pre-collision PDFs of one cell with plain global loads (AA odd: population i
// of x was stored by x - c_i in slot opp(i); otherwise slot i of x); with
// GHOST, populations entering from a ghost plane take the ghost value.
template <class S, int Q, int MODE, bool GHOST, class T>
__device__ __forceinline__ void psm_load(const StepParams& p, const Stencil& sn, const ZGhost& zg, unsigned cell,
                                         T (&f)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = lat_cx(i), cy = lat_cy(i), cz = lat_cz(i);
    if (GHOST && zg.from(cz)) {
      f[i] = cst<T>(p).ghost[i];
    } else if (MODE == MODE_AA_ODD) {
      f[i] = Store<S>::ld(static_cast<const S*>(p.src_slot[lat_opp(i)]) + sn.at(-cx, -cy, -cz));
    } else {
      f[i] = Store<S>::ld(static_cast<const S*>(p.src_slot[i]) + cell);
    }
  }
}

// Per-warp force/torque accumulation into s_ft[warp] (fixed order: warp
// butterfly in the contribution's precision, then added in FP64 in tile
// order).  All 32 lanes must call it.
template <class V>
__device__ __forceinline__ void warp_ft(double (*s_ft)[PSM_MAX_BODIES * 6], int nb, bool contributes, int owner,
                                        const V (&ft)[6]) {
  if (nb == 0 || !__any_sync(0xffffffffu, contributes)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int bi = 0; bi < nb; ++bi) {
    const bool mine = contributes && owner == bi;
    if (!__any_sync(0xffffffffu, mine)) continue;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const V v = warp_sum(mine ? ft[k] : V(0));
      if (lane == 0) s_ft[warp][bi * 6 + k] += (double)v;
    }
  }
}

// Block sum of the per-warp slots (fixed order), then the grid-wide ordered sum.
__device__ __forceinline__ void block_ft_finish(double (*s_ft)[PSM_MAX_BODIES * 6], const StepParams& p) {
  constexpr int NW = PSM_THREADS / 32;
  __shared__ double blk[PSM_MAX_BODIES * 6];
  const int ncomp = p.nbodies * 6;
  __syncthreads();
  if ((int)threadIdx.x < ncomp) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += s_ft[w][threadIdx.x];
    blk[threadIdx.x] = s;
  }
  __syncthreads();
  grid_reduce(blk, ncomp, p.partials, p.ticket, p.ft_out);
}

// Tile walk of a persistent block: tile index t = (z nty + ty) ntx + tx,
// advanced by the grid size without divisions after the first tile.
// (tile index t -> (tx, ty, z)) and its increment by a decomposed step
__device__ __forceinline__ int4 tile_split(const Tiling& t, int tile) {
  return make_int4(tile % t.ntx, (tile / t.ntx) % t.nty, tile / t.ntx / t.nty, 0);
}
__device__ __forceinline__ int4 tile_advance(const Tiling& t, int4 cur, int4 step) {
  cur.x += step.x;
  int c = cur.x >= t.ntx;
  cur.x -= c ? t.ntx : 0;
  cur.y += step.y + c;
  c = cur.y >= t.nty;
  cur.y -= c ? t.nty : 0;
  cur.z += step.z + c;
  return cur;
}

struct TileWalk {
  int tx, ty, z;       // current tile
  int gx, gy, gz;      // the grid size, decomposed like a tile index
  int ntx, nty;
  __device__ __forceinline__ void init(const Tiling& t, int tile, int step) {
    ntx = t.ntx;
    nty = t.nty;
    tx = tile % ntx;
    ty = (tile / ntx) % nty;
    z = tile / ntx / nty;
    gx = step % ntx;
    gy = (step / ntx) % nty;
    gz = step / ntx / nty;
  }
  __device__ __forceinline__ void advance() {
    tx += gx;
    int c = tx >= ntx;
    tx -= c ? ntx : 0;
    ty += gy + c;
    c = ty >= nty;
    ty -= c ? nty : 0;
    z += gz + c;
  }
};

// The bodies of this step, copied to shared memory at block start: from the
// launch parameters, or, for bodies whose motion the device integrates
// (two-way coupling), from device memory.  The caller synchronises the block.
__device__ __forceinline__ void load_bodies(const StepParams& p, DevBody* s_body) {
  static_assert(sizeof(DevBody) % 4 == 0, "DevBody is copied in 4-byte words");
  constexpr int W = (int)(sizeof(DevBody) / 4);
  for (int k = threadIdx.x; k < p.nbodies * W; k += blockDim.x) {
    const int b = k / W, w = k % W;
    const DevBody* src = ((p.free_mask >> b) & 1u) ? &p.dbody[b] : &p.body[b];
    reinterpret_cast<unsigned*>(&s_body[b])[w] = reinterpret_cast<const unsigned*>(src)[w];
  }
}

// A tile (TX x TY cells of one z plane) takes the fluid-only path when no
// body's cell box meets it, no eps perturbation is set and its plane is not
// next to a ghost plane: every cell of such a tile has B = 0, and no
// population of it enters or leaves through a ghost plane.
__device__ __forceinline__ bool tile_general(const StepParams& p, const DevBody* bodies, int x0, int y0, int z, int TX,
                                             int TY) {
  bool gen = p.delta != nullptr || (p.g.bc_z == PSM_BC_EQ_INLET_OUTLET && (z == 0 || z == p.g.nz - 1));
  const int zw = z + p.g.z0;  // world z of the plane (the body boxes are in world cells)
#pragma unroll
  for (int bi = 0; bi < PSM_MAX_BODIES; ++bi) {
    if (bi < p.nbodies) {
      const DevBody& b = bodies[bi];
      gen = gen || (x0 < b.x1 && x0 + TX > b.x0 && y0 < b.y1 && y0 + TY > b.y0 && zw >= b.z0 && zw < b.z1);
    }
  }
  return gen;
}

template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

// One cell of a fluid-only tile: moments and Omega^F (the arithmetic psm_collide
// takes for B = 0).
template <class T, int Q, int FL>
__device__ __forceinline__ void fluid_collide(const StepParams& p, T (&f)[Q]) {
  const ConstT<T>& C = cst<T>(p);
  T drho, rho, ux, uy, uz, uu;
  moments<T, Q>(f, C.rho0, drho, rho, ux, uy, uz, uu);
  fluid_relax<T, Q, FL>(C, f, drho, rho, ux, uy, uz, uu);
}

// ---------------------------------------------------------------------------
// The fused step kernel with plain global loads (any grid shape; persistent:
// blocks stride over tiles of TX x TY cells of one z plane).
// ---------------------------------------------------------------------------
template <class S, int Q, int MODE, int FL>
__global__ void __launch_bounds__(PSM_THREADS, step_min_blocks<S, Q, FL>())
    k_step(const __grid_constant__ StepParams p) {
  using T = typename Store<S>::T;
  __shared__ double s_ft[PSM_THREADS / 32][PSM_MAX_BODIES * 6];
  __shared__ DevBody s_body[PSM_MAX_BODIES];
  const int nb = p.nbodies;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = lane; k < PSM_MAX_BODIES * 6; k += 32) s_ft[warp][k] = 0.0;
  load_bodies(p, s_body);
  __syncthreads();

  const int ntiles = (int)p.t.ntiles;
  const int lx = (int)threadIdx.x % p.t.tx, ly = (int)threadIdx.x / p.t.tx;

  auto cell_body = [&](auto gen_c, int x, int y, int z) {
    constexpr bool GEN = decltype(gen_c)::value;
    const bool active = x < p.g.nx && y < p.g.ny;
    int owner = -1;
    bool solid_cell = false;
    ft_t<T> ft[6] = {0, 0, 0, 0, 0, 0};
    if (active) {
      const unsigned cell = ((unsigned)z * (unsigned)p.g.ny + (unsigned)y) * (unsigned)p.g.nx + (unsigned)x;
      Stencil sn;
      sn.init(p.g, x, y, z, cell);
      ZGhost zg;
      zg.init(p.g, z);
      T f[Q];
      psm_load<S, Q, MODE, GEN>(p, sn, zg, cell, f);
      if (GEN) psm_collide<T, Q, FL>(p, s_body, f, x, y, z + p.g.z0, cell, owner, solid_cell, ft);
      else fluid_collide<T, Q, FL>(p, f);
      if (MODE == MODE_AA_ODD) {
        // rebuild the stencil for the stores rather than keep it live through
        // the collision (register pressure); the empty asm hides the equality
        // of the inputs from common-subexpression elimination
        int xs = x, ys = y, zs = z;
        unsigned cs = cell;
        asm volatile("" : "+r"(xs), "+r"(ys), "+r"(zs), "+r"(cs));
        Stencil sn2;
        sn2.init(p.g, xs, ys, zs, cs);
        psm_store<S, Q, MODE, GEN>(p, sn2, zg, cs, f);
      } else {
        psm_store<S, Q, MODE, GEN>(p, sn, zg, cell, f);
      }
    }
    if (GEN) warp_ft(s_ft, nb, active && solid_cell && owner >= 0, owner, ft);
  };

  TileWalk walk;
  walk.init(p.t, blockIdx.x, gridDim.x);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, walk.advance()) {
    const int x0 = walk.tx * p.t.tx, y0 = walk.ty * p.t.ty, z = walk.z;
    if (tile_general(p, s_body, x0, y0, z, p.t.tx, p.t.ty)) cell_body(BoolC<true>{}, x0 + lx, y0 + ly, z);
    else cell_body(BoolC<false>{}, x0 + lx, y0 + ly, z);
  }
  if (nb == 0) return;
  block_ft_finish(s_ft, p);
}

// Most input stages of the TMA step kernel (the stage count follows from the
// shared memory per SM, see TmaLayout).
#ifndef PSM_TMA_MAX_STAGES
#define PSM_TMA_MAX_STAGES 8
#endif

__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
  return (unsigned)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// try_wait with a suspend-time hint: the thread may stop issuing until the
// phase completes or about `ns` nanoseconds have passed
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long* bar, unsigned parity, unsigned ns) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 P, [%1], %2, %3;\n selp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for a phase: one poll, then suspended polls until the phase
// completes, 100 ms pass (global timer) or 2^22 polls were made; false if the
// phase did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    if (globaltimer_ns() - t0 > 100000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const void* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_load_16(void* dst, const void* src, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void tma_store_4d(const void* map, int c0, int c1, int c2, int c3, const void* src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// output boxes per warp (AA even), where the shared memory allows it
#ifndef PSM_TMA_OUT_BUFS
#define PSM_TMA_OUT_BUFS 2
#endif


// Lattice components for a run-time direction index (the producer's copy
// jobs): c + 1 in two bits per direction.
__host__ __device__ constexpr unsigned long long lat_bits(int axis) {
  unsigned long long b = 0;
  for (int i = 0; i < 27; ++i)
    b |= (unsigned long long)((axis == 0 ? lat_cx(i) : (axis == 1 ? lat_cy(i) : lat_cz(i))) + 1) << (2 * i);
  return b;
}
constexpr unsigned long long kLatCX = lat_bits(0), kLatCY = lat_bits(1), kLatCZ = lat_bits(2);
__device__ __forceinline__ int lat_c_rt(unsigned long long bits, int i) { return (int)((bits >> (2 * i)) & 3ull) - 1; }

// Shared-memory layout of the TMA step kernel (bytes; every box 128-byte
// aligned): [barriers 128 B] [NST input stages] [NOUT output buffers].
//   input, own-cell modes (two-grid, AA even): one [Q][TY][TX] box per tile
//     (TX TY = 256 CPT): slot i of cell r of thread t at element
//     256 CPT i + 256 r + t;
//   input, AA odd (TX = 256, TY = 1): per direction i the 256 values of slot
//     opp(i) at x - c_i for the tile's cells at byte 128 + i ROW, preceded and
//     followed by a 16-byte x-edge chunk, so that cell lx reads element
//     lx - c_x of it with no branch;
//   output (AA even): per warp a [Q][32] box of its 32 cells (WBOX bytes),
//     written back by the warp's own TMA tensor store.
// The stage count NST fills the shared memory of the resident blocks the
// launch bounds aim at (228 KB per SM, less 1 KB per block reserved and the
// kernel's static shared memory), between 2 and PSM_TMA_MAX_STAGES: deeper
// pipelines for the narrower storage types keep more bytes in flight.  (The
// launch refuses a build whose static shared memory exceeds STATIC_SMEM.)
template <class S, int Q, int MODE, int FL = 0>
struct TmaLayout {
  static constexpr bool LOAD_OWN = MODE != MODE_AA_ODD;
  static constexpr bool STORE_TMA = PSM_TMA_STORE && MODE == MODE_AA_EVEN;
  // cells per thread and tile (tma_cells_per_thread: the host tiles alike)
  static constexpr int CPT = tma_cells_per_thread((int)sizeof(S), MODE, Q, FL);  // FL numbers the fluid like psm.h
  static constexpr int EP = 16 / (int)sizeof(S);  // elements per 16-byte edge chunk
  static constexpr int r128(int b) { return ((b + 127) / 128) * 128; }
  static constexpr int BOX_BYTES = Q * PSM_THREADS * CPT * (int)sizeof(S);
  static constexpr int BOX = r128(BOX_BYTES);
  // AA odd records: direction i's row of 256 values at byte 128 + i ROW of the
  // stage (128-byte aligned), its 16-byte edge chunks right before and after
  // it; ROW >= row + 32 bytes keeps the chunk after one row clear of the chunk
  // before the next (which sits in the last 16 bytes below that row)
  static constexpr int ROW = r128(PSM_THREADS * (int)sizeof(S) + 32);
  static constexpr int STAGE = LOAD_OWN ? BOX : r128(Q * ROW + 16);
  static constexpr int WBOX = r128(Q * 32 * (int)sizeof(S));
  static constexpr int OUT = STORE_TMA ? (PSM_THREADS / 32) * WBOX : 0;
  static constexpr int SM_SMEM = 233472;
  static constexpr int BLOCKS = step_min_blocks<S, Q, FL, MODE>();
  // per block: 1 KB reserved by the hardware and the kernel's static shared
  // memory (about 5 KB: force/torque slots, reduction scratch, the bodies of
  // the step, stage headers), allowed for with 6 KB
  static constexpr int STATIC_SMEM = 6144;
  static constexpr int BUDGET0 = (SM_SMEM - BLOCKS * (1024 + STATIC_SMEM)) / BLOCKS - 256;
  static constexpr int clamp_st(int n) { return n < 2 ? 2 : (n > PSM_TMA_MAX_STAGES ? PSM_TMA_MAX_STAGES : n); }
  // output boxes per warp: PSM_TMA_OUT_BUFS where that leaves at least 3 input stages, else 1
  static constexpr int NOUT = (PSM_TMA_OUT_BUFS > 1 && (BUDGET0 - PSM_TMA_OUT_BUFS * OUT) / STAGE >= 3) ? PSM_TMA_OUT_BUFS : 1;
  static constexpr int NST = clamp_st((BUDGET0 - NOUT * OUT) / STAGE);
  // + 128 B of barriers, + 128 B of alignment slack
  static constexpr int SMEM = 256 + NST * STAGE + NOUT * OUT;
};

// ---------------------------------------------------------------------------
// TMA-staged step kernel.  Shapes: tiles of TX x TY = 256 CPT cells of one z
// plane with nx % TX == 0 and ny % TY == 0 (TX = min(256, nx), a power of
// two), TX * sizeof(S) a multiple of 16 bytes; the AA odd step needs TX = 256.
// Persistent blocks stride over tiles.  Warp 0 keeps NST tiles of
// pre-collision PDFs in flight in shared memory (two-grid and AA even: one
// cp.async.bulk.tensor box per tile; AA odd: one row per direction plus
// 16-byte cp.async.bulk edge chunks for x - c_x) while all threads collide the
// oldest staged tile from shared memory.  The producer classifies each tile
// (tile_general) and the block takes the fluid-only path or the general one
// for the whole tile.  The two-grid and AA odd steps store to x + c_i with
// st.global; the AA even step stores to the own cells' swapped slots (with
// two cells per thread, the fluid-only tiles' x-neighbour pairs with one
// 32-bit access per slot), or, built with PSM_TMA_STORE, through one TMA
// tensor store per warp.  No block barrier inside the tile loop.
// ---------------------------------------------------------------------------
template <class S, int Q, int MODE, int FL>
__global__ void __launch_bounds__(PSM_THREADS, step_min_blocks<S, Q, FL, MODE>())
    k_step_tma(const __grid_constant__ StepParams p, const __grid_constant__ TmaMaps maps) {
  using T = typename Store<S>::T;
  using L = TmaLayout<S, Q, MODE, FL>;
  constexpr int NST = L::NST;
  constexpr int NOUT = L::NOUT;
  // refill lag in tiles: a stage is refilled LAG tiles after it was read, so the
  // refilling warp seldom waits for the slowest warp; NST - LAG tiles stay ahead
#ifdef PSM_TMA_REFILL_LAG
  constexpr int LAG = PSM_TMA_REFILL_LAG < NST - 1 ? PSM_TMA_REFILL_LAG : NST - 2;
#else
  constexpr int LAG = NST >= 5 ? 2 : (NST >= 3 ? 1 : 0);
#endif
  constexpr int EP = L::EP;
  __shared__ double s_ft[PSM_THREADS / 32][PSM_MAX_BODIES * 6];
  __shared__ int s_abort;
  __shared__ int s_issued[NST];  // loads issued per stage (warp 0, lane 0)
  __shared__ int4 s_hdr[NST];    // per stage: tile origin x0, y0, z and the general-path flag
  __shared__ DevBody s_body[PSM_MAX_BODIES];
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // dynamic shared memory is only guaranteed 16-byte alignment: align by hand
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  // barriers in the first 128 B: full[s] completes when stage s holds its tile
  // (the producer's arrival plus the copied bytes); empty[s] when every warp has
  // read it (one arrival per warp)
  unsigned long long* full = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* empty = full + NST;
  static_assert(2 * NST * 8 <= 128, "stage barriers exceed their 128 bytes");
  constexpr int NW = PSM_THREADS / 32;
  const int nb = p.nbodies;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = lane; k < PSM_MAX_BODIES * 6; k += 32) s_ft[warp][k] = 0.0;
  const int TX = p.t.tx, TY = p.t.ty;
  constexpr int CPT = L::CPT;
  if (TX * TY != PSM_THREADS * CPT) {
    // a tiling this instance was not built for: refuse before any wait or copy
    if (threadIdx.x == 0 && p.err) atomicExch(p.err, 2);
    return;
  }
  const int TYB = TY / CPT;  // rows of the tile covered by one cell per thread
  unsigned char* stages = base + 128;
  unsigned char* outs = stages + NST * L::STAGE;
  const int ntiles = (int)p.t.ntiles;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NW);
      s_issued[s] = 0;
    }
    fence_mbar_init();
  }
  load_bodies(p, s_body);
  __syncthreads();

  // producer: the 32 lanes of one warp stage the pre-collision PDFs of the
  // walk's current tile into stage `s`, one copy job per lane, and advance the
  // walk.  Warp 0 stages the first NST tiles; afterwards warp w refills the
  // stage of tile j when j = w (mod NW), so the producer work rotates over the
  // warps (its walk: tiles w + NST, w + NST + NW, ... of this block).
  // (kept in shared memory, not in registers across the tile loop)
  __shared__ int4 s_walk[NW];  // per warp: the next tile it refills (tx, ty, z)
  __shared__ int4 s_wstep;     // NW * gridDim.x, split like a tile index
  if (lane == 0) s_walk[warp] = tile_split(p.t, blockIdx.x + (warp + NST) * gridDim.x);
  if (threadIdx.x == 0) s_wstep = tile_split(p.t, NW * gridDim.x);
  __syncthreads();
  auto produce = [&](const int4 cur, int s) {
    const int z = cur.z;
    const int x0 = cur.x * TX, y0 = cur.y * TY;
    unsigned char* st = stages + s * L::STAGE;
    unsigned long long* bar = &full[s];
    fence_proxy_async();
    if (L::LOAD_OWN) {
      if (lane == 0) {
        mbar_expect_tx(bar, (unsigned)L::BOX_BYTES);
        tma_load_4d(st, &maps.tile, x0, y0, z, 0, bar);
      }
    } else {
      for (int i = lane; i < Q; i += 32) {
        const int cx = lat_c_rt(kLatCX, i), cy = lat_c_rt(kLatCY, i), cz = lat_c_rt(kLatCZ, i);
        int zs = z - cz;
        if (zs < 0 || zs >= p.g.nz) {
          if (p.g.bc_z == PSM_BC_EQ_INLET_OUTLET) continue;  // ghost populations: no load
          zs = zs < 0 ? zs + p.g.nz : zs - p.g.nz;
        }
        int ys = y0 - cy;
        ys = ys < 0 ? ys + p.g.ny : (ys >= p.g.ny ? ys - p.g.ny : ys);
        const int slot = lat_opp(i);
        unsigned char* row = st + i * L::ROW + 128;
        mbar_expect_tx(bar, (unsigned)(PSM_THREADS * (int)sizeof(S)));
        tma_load_4d(row, &maps.row1, x0, ys, zs, slot, bar);
        if (cx != 0) {
          // cx = +1: cell x0 reads x0 - 1 (the chunk before the row, wrapped in x);
          // cx = -1: cell x0 + 255 reads x0 + 256 (the chunk after it)
          const int xe = cx > 0 ? (x0 == 0 ? p.g.nx - EP : x0 - EP) : (x0 + PSM_THREADS == p.g.nx ? 0 : x0 + PSM_THREADS);
          // slot k starts k ncell values after slot 0 (one uniform base for every lane)
          const S* src = static_cast<const S*>(p.src_slot[0]) +
                         (((long long)slot * p.g.nz + zs) * p.g.ny + ys) * p.g.nx + xe;
          mbar_expect_tx(bar, 16u);
          bulk_load_16(cx > 0 ? row - 16 : row + PSM_THREADS * (int)sizeof(S), src, bar);
        }
      }
    }
    if (lane == 0) s_hdr[s] = make_int4(x0, y0, z, tile_general(p, s_body, x0, y0, z, TX, TY) ? 1 : 0);
    __syncwarp();  // every lane's expected bytes are registered before the arrival
    if (lane == 0) {
      mbar_arrive(bar);
      s_issued[s] += 1;
    }
  };

  if (warp == 0) {
    int4 first = tile_split(p.t, blockIdx.x);
    const int4 g1 = tile_split(p.t, gridDim.x);
    for (int k = 0; k < NST; ++k) {
      const int tile = blockIdx.x + k * gridDim.x;
      if (tile < ntiles) produce(first, k);
      first = tile_advance(p.t, first, g1);
    }
  }

  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int px = threadIdx.x % (TX / 2), py = threadIdx.x / (TX / 2);

  // One staged tile, read from stage s after its full barrier.  Each warp
  // signals empty[s] once it holds its cells' PDFs in registers; warp 0 then
  // waits for all warps' signals before refilling the stage, so warps do not
  // wait for one another otherwise.  A wait that times out sets s_abort and
  // the warp leaves the tile loop.
  // After the warp holds its cells' PDFs of stage s in registers.
  auto stage_read = [&](int tile, int k, int s) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    // refill the stage of tile j = k - LAG (read by every warp by now, as a
    // rule) with tile j + NST; warp j mod NW does it
    const int j = k - LAG;
    if (j >= 0 && warp == j % NW) {
      const int next = tile + (NST - LAG) * gridDim.x;
      if (next < ntiles) {
        const int sj = j % NST;
        // warp-uniform outcome (produce needs the whole warp)
        if (__all_sync(0xffffffffu, mbar_wait_bounded(&empty[sj], (unsigned)((j / NST) & 1)))) {
          const int4 cur = s_walk[warp];
          produce(cur, sj);
          if (lane == 0) s_walk[warp] = tile_advance(p.t, cur, s_wstep);
        } else {
          s_abort = 1;
        }
      }
    }
  };

  auto tile_body = [&](auto gen_c, int tile, int k, int s, const int4 hd) {
    constexpr bool GEN = decltype(gen_c)::value;
    const int z = hd.z;
    ZGhost zg;
    zg.init(p.g, z);
    const unsigned char* st = stages + s * L::STAGE;
    // fluid-only tiles of the AA even step in 16-bit storage: the thread's two
    // cells are x neighbours (x even, x + 1), so one 32-bit shared load and one
    // 32-bit store per slot serve both
    constexpr bool XPAIR = !GEN && CPT == 2 && MODE == MODE_AA_EVEN && sizeof(S) == 2 && FL != 2 && !L::STORE_TMA;
    if constexpr (XPAIR) {
      const unsigned* sw = reinterpret_cast<const unsigned*>(st) + (py * TX) / 2 + px;
      T f0[Q], f1[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) Pair16<S>::unpack(sw[i * (CPT * PSM_THREADS / 2)], f0[i], f1[i]);
      stage_read(tile, k, s);
      fluid_collide<T, Q, FL>(p, f0);
      fluid_collide<T, Q, FL>(p, f1);
      const int x = hd.x + 2 * px, y = hd.y + py;
      const unsigned cell = ((unsigned)z * (unsigned)p.g.ny + (unsigned)y) * (unsigned)p.g.nx + (unsigned)x;
#pragma unroll
      for (int i = 0; i < Q; ++i)
        *reinterpret_cast<unsigned*>(static_cast<S*>(p.dst_slot[lat_opp(i)]) + cell) = Pair16<S>::pack(f0[i], f1[i]);
      return;
    }
    // the thread's cells r = 0 .. CPT-1: (lx, ly + r TYB), one after the other
    auto one_cell = [&](int r) {
      const int x = hd.x + lx, y = hd.y + ly + r * TYB;
      const unsigned cell = ((unsigned)z * (unsigned)p.g.ny + (unsigned)y) * (unsigned)p.g.nx + (unsigned)x;
      T f[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (GEN && zg.from(lat_cz(i))) {
          f[i] = cst<T>(p).ghost[i];
        } else if (L::LOAD_OWN) {
          f[i] = Store<S>::ld(reinterpret_cast<const S*>(st) + (i * CPT + r) * PSM_THREADS + threadIdx.x);
        } else {
          f[i] = Store<S>::ld(reinterpret_cast<const S*>(st + i * L::ROW + 128) + (lx - lat_cx(i)));
        }
      }
      if (r == CPT - 1) stage_read(tile, k, s);
      int owner = -1;
      bool solid_cell = false;
      ft_t<T> ft[6] = {0, 0, 0, 0, 0, 0};
      if (GEN) psm_collide<T, Q, FL>(p, s_body, f, x, y, z + p.g.z0, cell, owner, solid_cell, ft);
      else fluid_collide<T, Q, FL>(p, f);
      if constexpr (L::STORE_TMA) {
        static_assert(CPT == 1, "TMA stores write one cell per thread");
        // this warp's output box of tile k; lane 0 issued (and committed) the
        // warp's earlier stores: the one NOUT tiles back must have read it
        S* ow = reinterpret_cast<S*>(outs + (k % NOUT) * L::OUT + warp * L::WBOX);
        if (lane == 0) bulk_wait_read<NOUT - 1>();
        __syncwarp();
#pragma unroll
        for (int i = 0; i < Q; ++i) Store<S>::st(ow + lat_opp(i) * 32 + lane, f[i]);
        fence_proxy_async();  // the generic-proxy writes above become visible to the TMA store
        __syncwarp();
        if (lane == 0) {
          const int w0 = warp * 32;
          tma_store_4d(&maps.dstw, hd.x + w0 % TX, hd.y + w0 / TX, z, 0, ow);
          bulk_commit();
        }
      } else {
        Stencil sn;
        sn.init(p.g, x, y, z, cell);
        psm_store<S, Q, MODE, GEN>(p, sn, zg, cell, f);
      }
      if (GEN) warp_ft(s_ft, nb, solid_cell && owner >= 0, owner, ft);
    };
    if constexpr (MODE == MODE_AA_EVEN) {
      // only general tiles come here (the fluid-only ones took the pairs above):
      // one copy of the PSM code
#pragma unroll 1
      for (int r = 0; r < CPT; ++r) one_cell(r);
    } else {
#pragma unroll
      for (int r = 0; r < CPT; ++r) one_cell(r);
    }
  };

  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int s = k % NST;
    // bounded wait for the stage, warp-uniform outcome (on time-out the block's
    // results are invalid: s_abort; the warp leaves the loop)
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (unsigned)((k / NST) & 1)))) {
      s_abort = 1;
      break;
    }
    const int4 hd = s_hdr[s];
    if (hd.w) tile_body(BoolC<true>{}, tile, k, s, hd);
    else tile_body(BoolC<false>{}, tile, k, s, hd);
  }
  if (L::STORE_TMA && lane == 0) bulk_wait_all();
  __syncthreads();
  if (s_abort) {
    if (threadIdx.x == 0) {
      if (p.err) atomicExch(p.err, 1);
      // let the copies already issued finish before the block's shared memory is released
      for (int s2 = 0; s2 < NST; ++s2)
        if (s_issued[s2] > 0) mbar_wait_bounded(&full[s2], (unsigned)((s_issued[s2] - 1) & 1));
    }
    __syncthreads();
  }
  if (nb == 0) return;
  block_ft_finish(s_ft, p);
}

// ---------------------------------------------------------------------------
// Import / export / diagnostics (one thread per cell of planes [z_begin, z_end))
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool io_cell(const IoParams& p, long long idx, int& x, int& y, int& z, long long& cell) {
  const long long plane = (long long)p.g.nx * p.g.ny;
  const long long n = plane * (p.z_end - p.z_begin);
  if (idx >= n) return false;
  z = p.z_begin + (int)(idx / plane);
  const long long r = idx % plane;
  y = (int)(r / p.g.nx);
  x = (int)(r % p.g.nx);
  cell = (long long)z * plane + r;
  return true;
}

// f_i(x) (shifted) of a state stored in `layout`, ghost value for populations
// entering from a ghost plane
template <class S, int Q>
__device__ __forceinline__ void read_state(const IoParams& p, const S* buf, const Nbr& nbr, long long cell,
                                           typename Store<S>::T f[Q]) {
  using T = typename Store<S>::T;
  const long long N = p.g.ncell;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (nbr.from_ghost(lat_cz(i))) {
      f[i] = T(p.ghost[i]);
    } else if (p.layout == LAYOUT_SWAPPED) {
      f[i] = Store<S>::ld(buf + (long long)lat_opp(i) * N +
                          (unsigned)((unsigned)cell + nbr.off(-lat_cx(i), -lat_cy(i), -lat_cz(i))));
    } else {
      f[i] = Store<S>::ld(buf + (long long)i * N + cell);
    }
  }
}

template <class S, int Q>
__global__ void k_import(const __grid_constant__ IoParams p) {
  S* buf = static_cast<S*>(p.f);
  const long long N = p.g.ncell;
  const long long plane = (long long)p.g.nx * p.g.ny;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;; idx += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    long long cell;
    if (!io_cell(p, idx, x, y, z, cell)) return;
    Nbr nbr;
    nbr.init(p.g, x, y, z);
    for (int i = 0; i < Q; ++i) {
      double v;
      if (p.uniform || p.rho_f) {
        const long long lc = cell - (long long)p.z_begin * plane;
        const double* uc = p.rho_f ? p.u_f + 3 * lc : p.u;
        const double rc = p.rho_f ? p.rho_f[lc] : p.rho;
        const double cu = lat_cx(i) * uc[0] + lat_cy(i) * uc[1] + lat_cz(i) * uc[2];
        const double uu = uc[0] * uc[0] + uc[1] * uc[1] + uc[2] * uc[2];
        v = lat_w<Q>(i) * rc * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
      } else {
        v = p.f_in[(long long)i * plane * (p.z_end - p.z_begin) + (cell - (long long)p.z_begin * plane)];
      }
      v -= lat_w<Q>(i) * p.rho0;
      if (nbr.from_ghost(lat_cz(i))) continue;  // such populations always read the ghost value
      long long dstc;
      int slot;
      if (p.layout == LAYOUT_SWAPPED) {
        slot = lat_opp(i);
        dstc = (unsigned)((unsigned)cell + nbr.off(-lat_cx(i), -lat_cy(i), -lat_cz(i)));
      } else {
        slot = i;
        dstc = cell;
      }
      buf[(long long)slot * N + dstc] = Store<S>::from_double(v);
    }
  }
}

template <class S, int Q>
__global__ void k_export(const __grid_constant__ IoParams p) {
  using T = typename Store<S>::T;
  const S* buf = static_cast<const S*>(p.f);
  const long long plane = (long long)p.g.nx * p.g.ny;
  const long long nchunk = plane * (p.z_end - p.z_begin);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;; idx += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    long long cell;
    if (!io_cell(p, idx, x, y, z, cell)) return;
    Nbr nbr;
    nbr.init(p.g, x, y, z);
    T f[Q];
    read_state<S, Q>(p, buf, nbr, cell, f);
    for (int i = 0; i < Q; ++i) p.f_out[(long long)i * nchunk + idx] = (double)f[i] + lat_w<Q>(i) * p.rho0;
  }
}

// Natural layout, shifted, storage precision (psm_get_pdfs): the stored
// values themselves (ghost-plane populations as the ghost value, rounded).
template <class S, int Q>
__global__ void k_export_raw(const __grid_constant__ IoParams p) {
  using T = typename Store<S>::T;
  const S* buf = static_cast<const S*>(p.f);
  S* out = static_cast<S*>(p.f_out_raw);
  const long long plane = (long long)p.g.nx * p.g.ny;
  const long long nchunk = plane * (p.z_end - p.z_begin);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;; idx += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    long long cell;
    if (!io_cell(p, idx, x, y, z, cell)) return;
    Nbr nbr;
    nbr.init(p.g, x, y, z);
    T f[Q];
    read_state<S, Q>(p, buf, nbr, cell, f);
    for (int i = 0; i < Q; ++i) Store<S>::st(out + (long long)i * nchunk + idx, f[i]);
  }
}

// Natural, unshifted FP64 PDFs of listed cells: out[k][Q].
template <class S, int Q>
__global__ void k_get_cells(const __grid_constant__ IoParams p, const long long* cells, long long n, double* out) {
  using T = typename Store<S>::T;
  const S* buf = static_cast<const S*>(p.f);
  const long long plane = (long long)p.g.nx * p.g.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long cell = cells[k];
    if (cell < 0 || cell >= p.g.ncell) continue;  // the host validates; never read out of bounds
    const int z = (int)(cell / plane);
    const long long r = cell % plane;
    const int y = (int)(r / p.g.nx), x = (int)(r % p.g.nx);
    Nbr nbr;
    nbr.init(p.g, x, y, z);
    T f[Q];
    read_state<S, Q>(p, buf, nbr, cell, f);
    for (int i = 0; i < Q; ++i) out[k * Q + i] = (double)f[i] + lat_w<Q>(i) * p.rho0;
  }
}

template <class S, int Q>
__global__ void k_macro(const __grid_constant__ IoParams p) {
  using T = typename Store<S>::T;
  const S* buf = static_cast<const S*>(p.f);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;; idx += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    long long cell;
    if (!io_cell(p, idx, x, y, z, cell)) return;
    Nbr nbr;
    nbr.init(p.g, x, y, z);
    T f[Q];
    read_state<S, Q>(p, buf, nbr, cell, f);
    double drho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      const double v = (double)f[i];
      drho += v;
      j[0] += lat_cx(i) * v;
      j[1] += lat_cy(i) * v;
      j[2] += lat_cz(i) * v;
    }
    const double rho = p.rho0 + drho;
    p.rho_out[idx] = rho;
    for (int k = 0; k < 3; ++k) p.u_out[3 * idx + k] = j[k] / rho;
  }
}

template <class S, int Q>
__global__ void __launch_bounds__(PSM_THREADS) k_mass(const __grid_constant__ IoParams p) {
  using T = typename Store<S>::T;
  const S* buf = static_cast<const S*>(p.f);
  double acc = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;; idx += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    long long cell;
    if (!io_cell(p, idx, x, y, z, cell)) break;
    Nbr nbr;
    nbr.init(p.g, x, y, z);
    T f[Q];
    read_state<S, Q>(p, buf, nbr, cell, f);
    double m = p.rho0;
    for (int i = 0; i < Q; ++i) m += (double)f[i];
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
  grid_reduce(blk, 1, p.partials, p.ticket, p.sum_out);
}

// ---------------------------------------------------------------------------
// Launcher helpers
// ---------------------------------------------------------------------------
template <class K>
int persistent_blocks(K kernel, long long work_blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, PSM_THREADS, 0);
  if (per_sm < 1) per_sm = 1;
  long long b = (long long)sms * per_sm;
  if (work_blocks < b) b = work_blocks;
  return (int)(b < 1 ? 1 : b);
}

template <class S, int Q, int MODE, int FL>
cudaError_t launch_step_t(const StepParams& p, cudaStream_t st) {
  static int blocks = persistent_blocks(k_step<S, Q, MODE, FL>, 1ll << 40);
  const int grid = (int)(p.t.ntiles < blocks ? p.t.ntiles : blocks);
  k_step<S, Q, MODE, FL><<<grid, PSM_THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

template <class S, int Q, int MODE, int FL>
cudaError_t launch_step_tma_t(const StepParams& p, const TmaMaps& m, cudaStream_t st) {
  using L = TmaLayout<S, Q, MODE, FL>;
  // persistent grid: resident blocks per SM (registers and shared memory), at most 8 per SM
  // The stage count assumes at most L::STATIC_SMEM bytes of static shared
  // memory per block; a build that exceeds it refuses to launch rather than
  // silently losing resident blocks.
  static const int blocks = [] {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_step_tma<S, Q, MODE, FL>) != cudaSuccess ||
        fa.sharedSizeBytes > (size_t)L::STATIC_SMEM)
      return 0;
    if (cudaFuncSetAttribute(k_step_tma<S, Q, MODE, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM) !=
        cudaSuccess)
      return 0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_tma<S, Q, MODE, FL>, PSM_THREADS, L::SMEM);
    if (per_sm > 8) per_sm = 8;
    return sms * per_sm;
  }();
  if (blocks < 1) return cudaErrorInvalidConfiguration;
  const long long grid = p.t.ntiles < blocks ? p.t.ntiles : blocks;
  k_step_tma<S, Q, MODE, FL><<<(int)grid, PSM_THREADS, L::SMEM, st>>>(p, m);
  return cudaGetLastError();
}

// fluid operator fl (PSM_BGK, PSM_TRT, PSM_CUMULANT) -> template argument FL;
// the cumulant kernels exist for D3Q19 only
template <class S, int Q, int MODE>
cudaError_t launch_step_tma_m(int fl, const StepParams& p, const TmaMaps& m, cudaStream_t st) {
  if (fl == PSM_TRT) return launch_step_tma_t<S, Q, MODE, 1>(p, m, st);
  if (fl == PSM_CUMULANT) {
    if constexpr (Q == 19) return launch_step_tma_t<S, Q, MODE, 2>(p, m, st);
    else return cudaErrorNotSupported;
  }
  return launch_step_tma_t<S, Q, MODE, 0>(p, m, st);
}

template <class S, int Q>
cudaError_t launch_step_tma_q(int mode, int fl, const StepParams& p, const TmaMaps& m, cudaStream_t st) {
  if (mode == MODE_TG) return launch_step_tma_m<S, Q, MODE_TG>(fl, p, m, st);
  if (mode == MODE_AA_EVEN) return launch_step_tma_m<S, Q, MODE_AA_EVEN>(fl, p, m, st);
  return launch_step_tma_m<S, Q, MODE_AA_ODD>(fl, p, m, st);
}

template <class S, int Q, int FL>
int tma_smem_f(int mode) {
  if (mode == MODE_TG) return TmaLayout<S, Q, MODE_TG, FL>::SMEM;
  if (mode == MODE_AA_EVEN) return TmaLayout<S, Q, MODE_AA_EVEN, FL>::SMEM;
  return TmaLayout<S, Q, MODE_AA_ODD, FL>::SMEM;
}

template <class S, int Q>
int tma_smem_q(int mode, int fl) {
  if constexpr (Q == 19)
    if (fl == PSM_CUMULANT) return tma_smem_f<S, Q, 2>(mode);
  return tma_smem_f<S, Q, 0>(mode);
}

// dynamic shared memory, stages, resident blocks aimed at, cells per thread
template <class L>
void tma_layout_of(int* out) {
  out[0] = L::SMEM;
  out[1] = L::NST;
  out[2] = L::BLOCKS;
  out[3] = L::CPT;
}
template <class S, int Q, int FL>
void tma_layout_f(int mode, int* out) {
  if (mode == MODE_TG) tma_layout_of<TmaLayout<S, Q, MODE_TG, FL>>(out);
  else if (mode == MODE_AA_EVEN) tma_layout_of<TmaLayout<S, Q, MODE_AA_EVEN, FL>>(out);
  else tma_layout_of<TmaLayout<S, Q, MODE_AA_ODD, FL>>(out);
}
template <class S, int Q>
void tma_layout_q(int mode, int fl, int* out) {
  if constexpr (Q == 19)
    if (fl == PSM_CUMULANT) return tma_layout_f<S, Q, 2>(mode, out);
  tma_layout_f<S, Q, 0>(mode, out);
}

template <class S, int Q, int MODE>
cudaError_t launch_step_m(int fl, const StepParams& p, cudaStream_t st) {
  if (fl == PSM_TRT) return launch_step_t<S, Q, MODE, 1>(p, st);
  if (fl == PSM_CUMULANT) {
    if constexpr (Q == 19) return launch_step_t<S, Q, MODE, 2>(p, st);
    else return cudaErrorNotSupported;
  }
  return launch_step_t<S, Q, MODE, 0>(p, st);
}

template <class S, int Q>
cudaError_t launch_step_q(int mode, int fl, const StepParams& p, cudaStream_t st) {
  if (mode == MODE_TG) return launch_step_m<S, Q, MODE_TG>(fl, p, st);
  if (mode == MODE_AA_EVEN) return launch_step_m<S, Q, MODE_AA_EVEN>(fl, p, st);
  return launch_step_m<S, Q, MODE_AA_ODD>(fl, p, st);
}

inline long long io_cells(const IoParams& p) { return (long long)p.g.nx * p.g.ny * (p.z_end - p.z_begin); }
inline int io_grid(const IoParams& p) {
  long long b = (io_cells(p) + PSM_THREADS - 1) / PSM_THREADS;
  if (b > 4096) b = 4096;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace psm

// One translation unit per storage precision defines its launchers with this.
#define PSM_DEFINE_STORAGE(NAME, S)                                                                     \
  namespace psm {                                                                                       \
  cudaError_t launch_step_##NAME(int Q, int mode, int fl, const StepParams& p, cudaStream_t st) {       \
    return Q == 19 ? launch_step_q<S, 19>(mode, fl, p, st) : launch_step_q<S, 27>(mode, fl, p, st);     \
  }                                                                                                     \
  cudaError_t launch_step_tma_##NAME(int Q, int mode, int fl, const StepParams& p, const TmaMaps& m,    \
                                     cudaStream_t st) {                                                 \
    return Q == 19 ? launch_step_tma_q<S, 19>(mode, fl, p, m, st) : launch_step_tma_q<S, 27>(mode, fl, p, m, st); \
  }                                                                                                     \
  int tma_smem_bytes_##NAME(int Q, int mode, int fl) {                                                  \
    return Q == 19 ? tma_smem_q<S, 19>(mode, fl) : tma_smem_q<S, 27>(mode, fl);                         \
  }                                                                                                     \
  void tma_layout_##NAME(int Q, int mode, int fl, int* out) {                                           \
    if (Q == 19) tma_layout_q<S, 19>(mode, fl, out);                                                    \
    else tma_layout_q<S, 27>(mode, fl, out);                                                            \
  }                                                                                                     \
  cudaError_t launch_import_##NAME(int Q, const IoParams& p, cudaStream_t st) {                         \
    if (Q == 19) k_import<S, 19><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                \
    else k_import<S, 27><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                        \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t launch_export_##NAME(int Q, const IoParams& p, cudaStream_t st) {                         \
    if (Q == 19) k_export<S, 19><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                \
    else k_export<S, 27><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                        \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t launch_export_raw_##NAME(int Q, const IoParams& p, cudaStream_t st) {                     \
    if (Q == 19) k_export_raw<S, 19><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                            \
    else k_export_raw<S, 27><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                    \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t launch_macro_##NAME(int Q, const IoParams& p, cudaStream_t st) {                          \
    if (Q == 19) k_macro<S, 19><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                 \
    else k_macro<S, 27><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                         \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t launch_get_cells_##NAME(int Q, const IoParams& p, const long long* cells, long long n,     \
                                      double* out, cudaStream_t st) {                                  \
    const int b = (int)((n + PSM_THREADS - 1) / PSM_THREADS < 1024 ? (n + PSM_THREADS - 1) / PSM_THREADS : 1024); \
    if (Q == 19) k_get_cells<S, 19><<<b < 1 ? 1 : b, PSM_THREADS, 0, st>>>(p, cells, n, out);         \
    else k_get_cells<S, 27><<<b < 1 ? 1 : b, PSM_THREADS, 0, st>>>(p, cells, n, out);                 \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t launch_mass_##NAME(int Q, const IoParams& p, int blocks, cudaStream_t st) {               \
    if (Q == 19) k_mass<S, 19><<<blocks, PSM_THREADS, 0, st>>>(p);                                      \
    else k_mass<S, 27><<<blocks, PSM_THREADS, 0, st>>>(p);                                              \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  }
