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

// ---------------------------------------------------------------------------
// Remap of one body onto one cell (Sec. 3).  The cell centre is taken into the
// body frame, X = Q_n^T (x_c - R_n), in float with a fixed order of separately
// rounded operations; the 2^s sub-cells per axis whose block starts at the
// sub-grid point nearest to X - 1/2 are counted in the brick-packed field.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long low_bits(int w) { return w >= 64 ? ~0ull : ((1ull << w) - 1ull); }

__device__ __forceinline__ float remap_eps(const DevBody& b, int x, int y, int z) {
  const int s = b.s;
  const int n = 1 << s;
  const float xc[3] = {__fadd_rn((float)x, 0.5f), __fadd_rn((float)y, 0.5f), __fadd_rn((float)z, 0.5f)};
  float d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = __fsub_rn(xc[k], b.Rf[k]);
  int a0[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float p0 = __fmul_rn(b.Qf[0 * 3 + k], d[0]);
    const float p1 = __fmul_rn(b.Qf[1 * 3 + k], d[1]);
    const float p2 = __fmul_rn(b.Qf[2 * 3 + k], d[2]);
    const float X = __fadd_rn(__fadd_rn(p0, p1), p2);
    const float t = __fsub_rn(X, b.Cf[k]);
    const float q = __fmul_rn(t, (float)n);
    a0[k] = (int)floorf(__fadd_rn(q, 0.5f));
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
  int count = 0;
  const int nn = n * n;
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
          // one word: bit (z n + y) n + x
          unsigned long long rowrep = 0, layrep = 0;
          for (int r = 0; r < nn; ++r) rowrep |= 1ull << (r * n);
          for (int l = 0; l < n; ++l) layrep |= 1ull << (l * nn);
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

// Eq. 3 (sign-corrected) minus the storage shift w rho0, for velocity v:
//   f^eq_i(rho, v) - w_i rho0 = w_i (drho + rho (3 c.v + 4.5 (c.v)^2 - 1.5 v.v))
template <int Q, class T>
__device__ __forceinline__ T feq_shifted(int i, T drho, T rho, T vx, T vy, T vz, T vv) {
  const T cv = T(lat_cx(i)) * vx + T(lat_cy(i)) * vy + T(lat_cz(i)) * vz;
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

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

template <class S, int Q, int MODE, int TRT>
__global__ void __launch_bounds__(PSM_THREADS, Q == 19 ? PSM_MIN_BLOCKS_Q19 : PSM_MIN_BLOCKS_Q27)
    k_step(const __grid_constant__ StepParams p) {
  using T = typename Store<S>::T;
  constexpr int NW = PSM_THREADS / 32;
  __shared__ double s_ft[NW][PSM_MAX_BODIES * 6];
  const int nb = p.nbodies;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = lane; k < PSM_MAX_BODIES * 6; k += 32) s_ft[warp][k] = 0.0;

  S* __restrict__ buf = static_cast<S*>(p.f);
  S* __restrict__ dst = static_cast<S*>(p.f_dst);
  const long long N = p.g.ncell;
  const T rho0 = T(p.rho0);
  const T om_a = T(p.om_a), om_b = T(p.om_b);
  const T inv_tau = T(1.0 / p.tau);

  const int ntiles = (int)p.t.ntiles;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int x, y, z;
    tile_coords(p.t, tile, x, y, z);
    const bool active = x < p.g.nx && y < p.g.ny;
    int owner = -1;
    bool solid_cell = false;
    double ft[6] = {0, 0, 0, 0, 0, 0};
    if (active) {
      const unsigned cell = ((unsigned)z * (unsigned)p.g.ny + (unsigned)y) * (unsigned)p.g.nx + (unsigned)x;
      Nbr nbr;
      nbr.init(p.g, x, y, z);
      // ---- load (pre-collision f, shifted) ----
      T f[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int cx = lat_cx(i), cy = lat_cy(i), cz = lat_cz(i);
        if (nbr.from_ghost(cz)) {
          f[i] = T(p.ghost[i]);
        } else if (MODE == MODE_AA_ODD) {
          f[i] = Store<S>::ld(buf + (long long)lat_opp(i) * N + (unsigned)(cell + nbr.off(-cx, -cy, -cz)));
        } else {
          f[i] = Store<S>::ld(buf + (long long)i * N + cell);
        }
      }
      // ---- remap (Sec. 3) and weighting (Eq. 5/6) ----
      const float epsf = cell_eps(p.body, nb, x, y, z, owner);
      T eps = T(epsf);
      if (p.delta) eps += T(p.delta[cell]);
      T Bw = eps;
      if (p.weighting == PSM_B_TAU_WEIGHTED) {
        const T t = T(p.tau - 0.5);
        Bw = eps * t / ((T(1) - eps) + t);
      }
      // ---- moments ----
      T drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        drho += f[i];
        if (lat_cx(i)) jx += T(lat_cx(i)) * f[i];
        if (lat_cy(i)) jy += T(lat_cy(i)) * f[i];
        if (lat_cz(i)) jz += T(lat_cz(i)) * f[i];
      }
      const T rho = rho0 + drho;
      const T inv_rho = T(1) / rho;
      const T ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
      const T uu = ux * ux + uy * uy + uz * uz;
      solid_cell = Bw != T(0);
      if (!solid_cell) {
        // ---- pure fluid: f* = f + Omega^F ----
        {
          const T n0 = f[0] - feq_shifted<Q, T>(0, drho, rho, ux, uy, uz, uu);
          f[0] = f[0] - (om_a + om_b) * n0;
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
          const int j = i + 1;
          const T ni = f[i] - feq_shifted<Q, T>(i, drho, rho, ux, uy, uz, uu);
          const T nj = f[j] - feq_shifted<Q, T>(j, drho, rho, ux, uy, uz, uu);
          if (TRT) {
            f[i] = f[i] - om_a * ni - om_b * nj;
            f[j] = f[j] - om_a * nj - om_b * ni;
          } else {
            f[i] = f[i] - om_a * ni;
            f[j] = f[j] - om_a * nj;
          }
        }
      } else {
        // ---- PSM cell: f* = f + (1 - B) Omega^F + B Omega^S (Eq. 4) ----
        T usx = 0, usy = 0, usz = 0;
        T rx = 0, ry = 0, rz = 0;
        if (owner >= 0) {
          const DevBody& b = p.body[owner];
          rx = T((double)x + 0.5 - b.R[0]);
          ry = T((double)y + 0.5 - b.R[1]);
          rz = T((double)z + 0.5 - b.R[2]);
          const T wx = T(b.omega[0]), wy = T(b.omega[1]), wz = T(b.omega[2]);
          usx = wy * rz - wz * ry + T(b.v[0]);
          usy = wz * rx - wx * rz + T(b.v[1]);
          usz = wx * ry - wy * rx + T(b.v[2]);
        }
        const T usus = usx * usx + usy * usy + usz * usz;
        const T omB = T(1) - Bw;
        T gx = 0, gy = 0, gz = 0;
        {
          const T n0 = f[0] - feq_shifted<Q, T>(0, drho, rho, ux, uy, uz, uu);
          const T m0 = f[0] - feq_shifted<Q, T>(0, drho, rho, usx, usy, usz, usus);
          const T of = -(om_a + om_b) * n0;
          T os;
          if (p.solid == PSM_SC1) os = n0 - m0;
          else if (p.solid == PSM_SC2) os = -m0 * inv_tau;
          else os = T(0);
          f[0] = f[0] + omB * of + Bw * os;
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
          const int j = i + 1;
          const T ni = f[i] - feq_shifted<Q, T>(i, drho, rho, ux, uy, uz, uu);
          const T nj = f[j] - feq_shifted<Q, T>(j, drho, rho, ux, uy, uz, uu);
          const T mi = f[i] - feq_shifted<Q, T>(i, drho, rho, usx, usy, usz, usus);
          const T mj = f[j] - feq_shifted<Q, T>(j, drho, rho, usx, usy, usz, usus);
          const T ofi = TRT ? (-om_a * ni - om_b * nj) : (-om_a * ni);
          const T ofj = TRT ? (-om_a * nj - om_b * ni) : (-om_a * nj);
          T osi, osj;
          if (p.solid == PSM_SC1) {
            osi = nj - mi;
            osj = ni - mj;
          } else if (p.solid == PSM_SC2) {
            osi = -mi * inv_tau;
            osj = -mj * inv_tau;
          } else {
            osi = mj - mi;
            osj = mi - mj;
          }
          f[i] = f[i] + omB * ofi + Bw * osi;
          f[j] = f[j] + omB * ofj + Bw * osj;
          // c_j = -c_i: sum_i Omega^S_i c_i over the pair
          const T d = osi - osj;
          if (lat_cx(i)) gx += T(lat_cx(i)) * d;
          if (lat_cy(i)) gy += T(lat_cy(i)) * d;
          if (lat_cz(i)) gz += T(lat_cz(i)) * d;
        }
        if (owner >= 0) {
          // Eq. 10 / 11 per cell; the body receives minus the solid's momentum transfer
          const double Gx = (double)(Bw * gx), Gy = (double)(Bw * gy), Gz = (double)(Bw * gz);
          const DevBody& b = p.body[owner];
          const double Rx = (double)x + 0.5 - b.R[0], Ry = (double)y + 0.5 - b.R[1], Rz = (double)z + 0.5 - b.R[2];
          ft[0] = -Gx;
          ft[1] = -Gy;
          ft[2] = -Gz;
          ft[3] = -(Ry * Gz - Rz * Gy);
          ft[4] = -(Rz * Gx - Rx * Gz);
          ft[5] = -(Rx * Gy - Ry * Gx);
        }
      }
      // ---- streamed store (Eq. 1) ----
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int cx = lat_cx(i), cy = lat_cy(i), cz = lat_cz(i);
        if (MODE == MODE_AA_EVEN) {
          Store<S>::st(buf + (long long)lat_opp(i) * N + cell, f[i]);
        } else if (!nbr.to_ghost(cz)) {
          S* base = (MODE == MODE_TG) ? dst : buf;
          Store<S>::st(base + (long long)i * N + (unsigned)(cell + nbr.off(cx, cy, cz)), f[i]);
        }
      }
    }
    // ---- per-warp force/torque accumulation (fixed order) ----
    if (nb > 0) {
      const bool contributes = active && solid_cell && owner >= 0;
      if (__any_sync(0xffffffffu, contributes)) {
        for (int bi = 0; bi < nb; ++bi) {
          const bool mine = contributes && owner == bi;
          if (!__any_sync(0xffffffffu, mine)) continue;
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const double v = warp_sum(mine ? ft[k] : 0.0);
            if (lane == 0) s_ft[warp][bi * 6 + k] += v;
          }
        }
      }
    }
  }
  if (nb == 0) return;
  __syncthreads();
  __shared__ double blk[PSM_MAX_BODIES * 6];
  const int ncomp = nb * 6;
  if ((int)threadIdx.x < ncomp) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += s_ft[w][threadIdx.x];
    blk[threadIdx.x] = s;
  }
  __syncthreads();
  grid_reduce(blk, ncomp, p.partials, p.ticket, p.ft_out);
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
      if (p.uniform) {
        const double cu = lat_cx(i) * p.u[0] + lat_cy(i) * p.u[1] + lat_cz(i) * p.u[2];
        const double uu = p.u[0] * p.u[0] + p.u[1] * p.u[1] + p.u[2] * p.u[2];
        v = lat_w<Q>(i) * p.rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
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

template <class S, int Q, int MODE, int TRT>
cudaError_t launch_step_t(const StepParams& p, cudaStream_t st) {
  static int blocks = persistent_blocks(k_step<S, Q, MODE, TRT>, 1ll << 40);
  const int grid = (int)(p.t.ntiles < blocks ? p.t.ntiles : blocks);
  k_step<S, Q, MODE, TRT><<<grid, PSM_THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

template <class S, int Q, int MODE, int TRT>
int step_blocks_t() {
  static int blocks = persistent_blocks(k_step<S, Q, MODE, TRT>, 1ll << 40);
  return blocks;
}

template <class S, int Q>
cudaError_t launch_step_q(int mode, int trt, const StepParams& p, cudaStream_t st) {
  if (mode == MODE_TG) return trt ? launch_step_t<S, Q, MODE_TG, 1>(p, st) : launch_step_t<S, Q, MODE_TG, 0>(p, st);
  if (mode == MODE_AA_EVEN)
    return trt ? launch_step_t<S, Q, MODE_AA_EVEN, 1>(p, st) : launch_step_t<S, Q, MODE_AA_EVEN, 0>(p, st);
  return trt ? launch_step_t<S, Q, MODE_AA_ODD, 1>(p, st) : launch_step_t<S, Q, MODE_AA_ODD, 0>(p, st);
}

template <class S, int Q>
int step_blocks_q(int mode, int trt) {
  if (mode == MODE_TG) return trt ? step_blocks_t<S, Q, MODE_TG, 1>() : step_blocks_t<S, Q, MODE_TG, 0>();
  if (mode == MODE_AA_EVEN) return trt ? step_blocks_t<S, Q, MODE_AA_EVEN, 1>() : step_blocks_t<S, Q, MODE_AA_EVEN, 0>();
  return trt ? step_blocks_t<S, Q, MODE_AA_ODD, 1>() : step_blocks_t<S, Q, MODE_AA_ODD, 0>();
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
  cudaError_t launch_step_##NAME(int Q, int mode, int trt, const StepParams& p, cudaStream_t st) {      \
    return Q == 19 ? launch_step_q<S, 19>(mode, trt, p, st) : launch_step_q<S, 27>(mode, trt, p, st);   \
  }                                                                                                     \
  int step_grid_blocks_##NAME(int Q, int mode, int trt) {                                               \
    return Q == 19 ? step_blocks_q<S, 19>(mode, trt) : step_blocks_q<S, 27>(mode, trt);                 \
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
  cudaError_t launch_macro_##NAME(int Q, const IoParams& p, cudaStream_t st) {                          \
    if (Q == 19) k_macro<S, 19><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                 \
    else k_macro<S, 27><<<io_grid(p), PSM_THREADS, 0, st>>>(p);                                         \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  cudaError_t launch_mass_##NAME(int Q, const IoParams& p, int blocks, cudaStream_t st) {               \
    if (Q == 19) k_mass<S, 19><<<blocks, PSM_THREADS, 0, st>>>(p);                                      \
    else k_mass<S, 27><<<blocks, PSM_THREADS, 0, st>>>(p);                                              \
    return cudaGetLastError();                                                                          \
  }                                                                                                     \
  }
