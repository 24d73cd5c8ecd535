// Internal declarations shared by the host API (psm_api.cu) and the kernel
// translation units (psm_kern_*.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/psm.h"

namespace psm {

enum Storage { ST_FP64 = PSM_FP64, ST_FP32 = PSM_FP32, ST_FP16 = PSM_FP16_SHIFTED, ST_BF16 = PSM_BF16_SHIFTED };

// Access pattern of one step kernel.
//   MODE_TG      : two grids, push: read own slot i (natural), write slot i of
//                  x + c_i in the other buffer (natural);
//   MODE_AA_EVEN : read own slot i (natural), write own slot opp(i) (swapped);
//   MODE_AA_ODD  : read slot opp(i) of x - c_i (swapped), write slot i of
//                  x + c_i (natural).
enum Mode { MODE_TG = 0, MODE_AA_EVEN = 1, MODE_AA_ODD = 2 };

// 1: the AA even step of the TMA kernel writes its tiles back with TMA tensor
// stores (one per warp); 0 (default, measured faster on GB300): plain stores
#ifndef PSM_TMA_STORE
#define PSM_TMA_STORE 0
#endif
// Cells per thread in a tile of the TMA step kernel: PSM_TMA_CPT16 for the
// D3Q19 two-grid step and the D3Q19 and D3Q27 AA even steps with BGK/TRT in
// 2-byte storage (FP16, BF16), where the kernel is issue-bound and sharing
// the per-tile work (stage wait, refill, tile classification, loop) between
// two cells measured faster (in the AA even step the two cells of a
// fluid-only tile are x neighbours: one 32-bit shared load and one 32-bit
// store per slot serve both); one elsewhere (memory-bound 4- and 8-byte
// storage; the D3Q27 two-grid step, the AA odd step and the cumulant, where
// the larger stages of two-cell tiles cost more pipeline depth than the
// shared work saves).
#ifndef PSM_TMA_CPT16
#define PSM_TMA_CPT16 2
#endif
__host__ __device__ constexpr int tma_cells_per_thread(int storage_bytes, int mode, int Q, int fluid) {
  return (storage_bytes == 2 && fluid != PSM_CUMULANT && ((mode == MODE_TG && Q == 19) || mode == MODE_AA_EVEN))
             ? PSM_TMA_CPT16
             : 1;
}

// Layout a state is stored in.  Pre-collision f_i(x) sits at
//   NATURAL: slot i of x;  SWAPPED: slot opp(i) of x - c_i.
// Populations whose upstream cell x - c_i lies in a ghost plane are not
// stored in either layout: they take the ghost value.
enum Layout { LAYOUT_NATURAL = 0, LAYOUT_SWAPPED = 1 };

// One body as the kernels see it at one step.
struct DevBody {
  const unsigned long long* bricks;  // [gz][gy][gx][wpb] words
  // occupancy [gz + 1][gy + 1][gx + 1] bytes, index c + 1 for c = -1 .. g - 1 per
  // axis: non-zero iff a brick in {c, c + 1}^3 has a set bit (nullptr: none)
  const unsigned char* occ;
  // occupancy of blocks of 8^3 occupancy cells, one bit each (index
  // (bz o8y + by) o8x + bx for occupancy index c + 1 = 8 b + 0..7 per axis):
  // set iff an occupancy byte of the block is (nullptr: none); a small array
  // that stays in L1, tested before the occupancy byte itself
  const unsigned* occ8;
  int o8x, o8y;
  int gx, gy, gz;
  int s;    // super-sampling depth
  int wpb;  // 64-bit words per brick
  // Pose of this step for the remap (Sec. 3).  The sub-cell block of a cell
  // starts at a0_k = floor(((X_k - 1/2) - lo_k) 2^s + 1/2), X = Q^T (x_c - R),
  // evaluated in double with separately rounded operations in that order.
  // The kernels decide it from the float form below and fall back to that
  // double evaluation for cells whose float value lies within rtol of a
  // decision boundary (remap_setup, remap_eps).
  double Qd[9];  // world <- body, row-major
  double lod[3];  // geometry box origin (body frame)
  // r_k = sum_j G_jk e_j + H_k with e = x - anchor, G = 2^s Q and H a constant
  // of the pose; the high parts are exact in float for every cell of the box
  float Ghi[9], Glo[9];  // [j * 3 + k]
  float Hhi[3], Hlo[3];
  int anchor[3];
  float rtol;     // bound on |r_float - r_double| over the box (2: always double)
  float Rf[3];    // reference point R_n rounded to float (FP32 lever arm)
  // kinematics in double (FP64 path, force/torque lever arm) and float (FP32 path)
  double R[3];
  double omega[3];
  double v[3];
  float omegaf[3];
  float vf[3];
  // cells tested for this body: [x0, x1) x [y0, y1) x [z0, z1), world cell indices
  int x0, x1, y0, y1, z0, z1;
};

// Float form of the remap's sub-cell decision for the pose (Q, R) of one
// body and its bound, for the cells of the box [x0, x1) x [y0, y1) x [z0, z1)
// set in d.  With an anchor cell a of the box, e = x - a and c = a + 1/2 - R,
//   r_k = ((X_k - 1/2) - lo_k) 2^s + 1/2 = sum_j G_jk e_j + H_k,
//   G = 2^s Q,  H_k = ((sum_j Q_jk c_j - 1/2) - lo_k) 2^s + 1/2.
// G and H split into high parts on the grid 2^-m and float low parts; m is
// the finest grid on which |H_hi| + sum_j |G_hi,jk| |e_j| stays below 2^(24-m)
// over the box, so that every product and partial sum of the high parts is a
// float exactly.  rtol bounds (twice, plus one float rounding of the distance
// test) the first-order errors of the float evaluation (rounding of G_lo and
// H_lo, three fma roundings of the low sum, one of the final add), of the
// double evaluation against exact arithmetic, and of H itself.
__host__ __device__ inline void remap_setup(DevBody& d, const double Q[9], const double R[3], const double lo[3]) {
  const double n = (double)(1 << d.s);
  const double U = 5.9604644775390625e-08;    // 2^-24, float unit round-off
  const double Ud = 1.1102230246251565e-16;   // 2^-53, double unit round-off
  const int b0[3] = {d.x0, d.y0, d.z0}, b1[3] = {d.x1, d.y1, d.z1};
  double Be = 0.0, Bd = 0.0, lom = 0.0;  // sum_j max |e_j|, sum_j max |x_j + 1/2 - R_j|, max |lo_k|
  for (int j = 0; j < 3; ++j) {
    const int last = b1[j] > b0[j] ? b1[j] - 1 : b0[j];
    d.anchor[j] = b0[j] + (last - b0[j]) / 2;
    Be += fmax(fabs((double)(b0[j] - d.anchor[j])), fabs((double)(last - d.anchor[j])));
    Bd += fmax(fabs((double)b0[j] + 0.5 - R[j]), fabs((double)last + 0.5 - R[j]));
    lom = fmax(lom, fabs(lo[j]));
  }
  for (int k = 0; k < 9; ++k) d.Qd[k] = Q[k];
  double H[3], Hmax = 0.0;
  for (int k = 0; k < 3; ++k) {
    d.lod[k] = lo[k];
    double X = 0.0;
    for (int j = 0; j < 3; ++j) X += Q[3 * j + k] * (((double)d.anchor[j] + 0.5) - R[j]);
    H[k] = ((X - 0.5) - lo[k]) * n + 0.5;
    Hmax = fmax(Hmax, fabs(H[k]));
  }
  const double span = (Hmax + 1.0) + (n + 1.0) * Be;
  int m = 20;
  while (m >= 0 && span * (double)(1 << m) >= 16777216.0) --m;
  if (m < 0 || !(span < 1e30)) {  // no exact float form: every cell takes the double decision
    for (int k = 0; k < 9; ++k) d.Ghi[k] = d.Glo[k] = 0.0f;
    for (int k = 0; k < 3; ++k) d.Hhi[k] = d.Hlo[k] = 0.0f;
    d.rtol = 2.0f;  // above any distance to the nearest integer (<= 1/2)
    return;
  }
  const double sc = (double)(1 << m), isc = 1.0 / sc;
  for (int k = 0; k < 9; ++k) {
    const double G = Q[k] * n;                     // exact (power of two)
    const double gh = floor(G * sc + 0.5) * isc;   // on the grid 2^-m, |gh| 2^m < 2^24
    d.Ghi[k] = (float)gh;
    d.Glo[k] = (float)(G - gh);
  }
  for (int k = 0; k < 3; ++k) {
    const double hh = floor(H[k] * sc + 0.5) * isc;
    d.Hhi[k] = (float)hh;
    d.Hlo[k] = (float)(H[k] - hh);
  }
  const double L = 0.5 * isc * (1.0 + Be);                  // bound on |low sum| and its partials
  const double ef = U * 0.5 * isc * (1.0 + Be) + 3.0 * U * L + U * (1.0 + L);
  const double ed = n * Ud * (7.0 * Bd + 3.0 * lom + 2.0) + Ud;  // double evaluation vs exact
  d.rtol = (float)(2.0 * (ef + 2.0 * ed) + U);
}

// State of a body moving under the fluid's force and torque (two-way
// coupling), integrated on the device after every step (FP64).
struct BodyDyn {
  double R[3], v[3], Q[9], w[3], L[3];  // position, velocity, orientation (world <- body), omega, L
  double mass, Ibinv[9];                // mass, inverse body-frame inertia
  double Fext[3], Text[3];              // constant external force and torque (world)
  double lo[3];                         // geometry box origin (body frame)
  int gx, gy, gz;                       // geometry box size (cells)
};

struct Grid3 {
  int nx, ny, nz;
  long long ncell;
  int bc_z;  // PSM_BC_PERIODIC / PSM_BC_EQ_INLET_OUTLET
  int z0;    // world z of plane 0 (a z-slab of a larger domain; 0 otherwise): cell centres are
             // (x + 1/2, y + 1/2, z + z0 + 1/2) for the remap, u_s and the torque lever arm
};

struct Tiling {
  int tx, ty;    // threads per block along x, y (tx * ty = PSM_THREADS)
  int ntx, nty;  // tiles along x, y
  long long ntiles;
};

// Per-step constants in the compute precision, precomputed on the host so that
// no kernel converts or divides doubles per cell.
template <class T>
struct ConstT {
  T rho0;
  T om_a, om_b;  // TRT as Omega^F_i = -om_a n_i - om_b n_opp(i); BGK: om_a = 1/tau, om_b = 0
  T inv_tau;     // 1 / tau (SC2)
  T tmh;         // tau - 1/2 (Eq. 6)
  T ghost[27];   // shifted ghost-plane populations f^eq_i(rho0, u_in) - w_i rho0
  // fluid collision (fluid_relax): omega+ = om_a + om_b, omega- = om_a - om_b,
  // and per weight class c = |c_i|^2 with weight w_c:
  T omp1, hp1, hm1;  // 1 - omega+, (1 - omega+) / 2, (1 - omega-) / 2
  T pw[4];        // omega+ w_c
  T pk[4];        // 4.5 omega+ w_c
  T pd[4];        // 3 omega- w_c
  T cum1[4];      // cumulant: 1 - omega for shear (1/tau), bulk, third order, fourth order
  int cum_unit;   // cumulant: bulk, third- and fourth-order rates all 1
};

struct StepParams {
  Grid3 g;
  Tiling t;
  void* f;      // AA: the buffer; TG: source
  void* f_dst;  // TG: destination
  // slot base pointers (set_slots): src_slot[i] = f + i ncell, dst_slot[i] =
  // (TG: f_dst, AA: f) + i ncell, in elements of the storage type; read from
  // the parameter bank, so a streamed access costs one 32-bit index and one
  // address computation
  void* src_slot[27];
  void* dst_slot[27];
  int fluid;      // PSM_BGK, PSM_TRT, PSM_CUMULANT
  int solid;      // 1, 2, 3
  int weighting;  // 0 direct, 1 tau-weighted
  int nbodies;
  DevBody body[PSM_MAX_BODIES];
  // bodies whose motion the device integrates (two-way coupling): bit b set ->
  // body b of this step is dbody[b] (device memory), not body[b]
  unsigned free_mask;
  const DevBody* dbody;
  const float* delta;  // optional additive eps perturbation per cell (nullptr: none)
  // force/torque reduction
  double* partials;      // [gridDim.x][nbodies * 6]
  unsigned int* ticket;  // zero between launches
  double* ft_out;        // [nbodies * 6] of this step (body convention)
  int* err;              // set non-zero by a kernel that gave up waiting (never traps)
  ConstT<float> cf;      // constants for FP32 arithmetic
  ConstT<double> cd;     // constants for FP64 arithmetic
};

// Tensor maps of the PDF buffers viewed as 4-D tensors (x, y, z, slot) for one
// launch of the TMA step kernel.
struct TmaMaps {
  CUtensorMap tile;  // source buffer, box (TX, TY, 1, Q): all slots of one tile
  CUtensorMap row1;  // source buffer, box (TX, 1, 1, 1): one slot of one row
  CUtensorMap dstw;  // destination of the AA even step's per-warp TMA stores, box (32, 1, 1, Q)
};

// Parameters of the import / export / reduction kernels.
struct IoParams {
  Grid3 g;
  Tiling t;
  void* f;
  int layout;  // Layout
  double ghost[27];
  double rho0;
  int z_begin, z_end;  // z-planes handled by this launch
  // import: from a natural FP64 state chunk (f_in, planes z_begin..z_end), uniform
  // (rho, u), or equilibria of per-cell fields (rho_f[cell], u_f[cell][3] of the chunk)
  const double* f_in;
  int uniform;
  double rho, u[3];
  const double* rho_f;
  const double* u_f;
  // export
  double* f_out;    // natural, unshifted, planes z_begin..z_end
  void* f_out_raw;  // natural, shifted, storage precision, planes z_begin..z_end
  double* rho_out;  // macroscopic
  double* u_out;
  // reduction
  double* partials;
  unsigned int* ticket;
  double* sum_out;
};

// Parameters of the stand-alone remap kernel (psm_get_eps).
struct RemapParams {
  Grid3 g;
  Tiling t;
  int nbodies;
  DevBody body[PSM_MAX_BODIES];
  int z_begin, z_end;
  float* eps_out;
};

constexpr int PSM_THREADS = 256;

// Caller-owned memory: PSM_OK when p points into device memory of the current
// device (or managed memory) with at least `bytes` bytes from p to the end of
// its allocation (the allocation's extent is checked where the driver reports
// it); otherwise PSM_ERR_ARG with a message naming `what`.  Launches nothing.
int check_device_buffer(const void* p, size_t bytes, const char* what);

Tiling make_tiling(int nx, int ny, int nz);
// fills p.src_slot / p.dst_slot from p.f, p.f_dst (nullptr: in place), p.g.ncell
void set_slots(StepParams& p, int storage, int Q);

// Launchers (one set per storage precision, in psm_kern_<storage>.cu).  Each
// returns cudaSuccess or the launch error.  `grid_out` reports the number of
// blocks the step kernel uses (so the host sizes the partials array).
cudaError_t launch_step(int storage, int Q, int mode, const StepParams& p, cudaStream_t st);
// TMA-staged variant (shape rules at k_step_tma); p.t must be the TMA tiling.
cudaError_t launch_step_tma(int storage, int Q, int mode, const StepParams& p, const TmaMaps& m, cudaStream_t st);
// dynamic shared memory bytes of the TMA variant for one mode
int tma_smem_bytes(int storage, int Q, int mode, int fl);
cudaError_t launch_import(int storage, int Q, const IoParams& p, cudaStream_t st);
cudaError_t launch_export(int storage, int Q, const IoParams& p, cudaStream_t st);
cudaError_t launch_export_raw(int storage, int Q, const IoParams& p, cudaStream_t st);
cudaError_t launch_macro(int storage, int Q, const IoParams& p, cudaStream_t st);
cudaError_t launch_mass(int storage, int Q, const IoParams& p, int blocks, cudaStream_t st);
cudaError_t launch_remap(const RemapParams& p, cudaStream_t st);
// one rigid-body step of the bodies in `mask` from the force/torque series
// entry ft (this step's) -> their DevBody of the next step
cudaError_t launch_body_update(BodyDyn* dyn, DevBody* dev, const double* ft, unsigned mask, int nb, int nx, int ny,
                               int nz, cudaStream_t st);
// occupancy of a geometry field (DevBody::occ) from its bricks (device)
cudaError_t launch_occupancy(const unsigned long long* bricks, int gx, int gy, int gz, int wpb, unsigned char* occ,
                             cudaStream_t st);
// block occupancy bits (DevBody::occ8, zeroed by the caller) from the occupancy
// bytes of a (gx + 1) x (gy + 1) x (gz + 1) array
cudaError_t launch_occupancy8(const unsigned char* occ, int ox, int oy, int oz, unsigned* occ8, cudaStream_t st);

#define PSM_DECLARE_STORAGE(NAME)                                                          \
  cudaError_t launch_step_##NAME(int Q, int mode, int fl, const StepParams& p, cudaStream_t st); \
  cudaError_t launch_step_tma_##NAME(int Q, int mode, int fl, const StepParams& p, const TmaMaps& m, \
                                     cudaStream_t st);                                    \
  int tma_smem_bytes_##NAME(int Q, int mode, int fl);                                             \
  void tma_layout_##NAME(int Q, int mode, int fl, int* out);                                      \
  cudaError_t launch_import_##NAME(int Q, const IoParams& p, cudaStream_t st);            \
  cudaError_t launch_export_##NAME(int Q, const IoParams& p, cudaStream_t st);            \
  cudaError_t launch_export_raw_##NAME(int Q, const IoParams& p, cudaStream_t st);        \
  cudaError_t launch_macro_##NAME(int Q, const IoParams& p, cudaStream_t st);             \
  cudaError_t launch_mass_##NAME(int Q, const IoParams& p, int blocks, cudaStream_t st);  \
  cudaError_t launch_get_cells_##NAME(int Q, const IoParams& p, const long long* cells, long long n, double* out, \
                                      cudaStream_t st);

PSM_DECLARE_STORAGE(fp64)
PSM_DECLARE_STORAGE(fp32)
PSM_DECLARE_STORAGE(fp16)
PSM_DECLARE_STORAGE(bf16)

}  // namespace psm
