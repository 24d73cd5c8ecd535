/*
 * psm.h -- C ABI of libpsm: the Partially Saturated Cells Method (PSM)
 * lattice Boltzmann hot path on one NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2502.20049.  One time step n of a solver handle is
 *   1. the pose of every body at step n (Sec. 3: rotation of the cell centre
 *      into the body frame, plus a translation),
 *   2. the remap of the super-sampled binary geometry field onto the per-cell
 *      solid fraction eps (Sec. 3),
 *   3. the per-cell PSM collision f* = f + (1 - B) Omega^F + B Omega^S
 *      (Eq. 4) with Omega^F = BGK (Eq. 2), TRT or cumulant, Omega^S = SC1/SC2/SC3
 *      (Eq. 7/8/9), B = B(eps) (Eq. 5 or Eq. 6), f^eq of Eq. 3 (read with
 *      -u.u/(2 c_s^2)),
 *   4. streaming f_i(x + c_i, t + 1) = f*_i(x) (Eq. 1): AA pattern in place, or
 *      two grids,
 *   5. the force and torque on every body (Eq. 10 and Eq. 11), reduced in FP64.
 * It runs fused in one kernel launch per step.
 *
 * Conventions:
 *   - lattice units dx = dt = 1; cell (x, y, z) has its centre at
 *     (x + 1/2, y + 1/2, z + 1/2);
 *   - PDF arrays are [Q][nz][ny][nx] (x fastest), in the direction order that
 *     psm_lattice_velocities() returns;
 *   - x and y are periodic; z is periodic or bounded by two equilibrium ghost
 *     planes holding f^eq(rho0, u_in) (populations entering from a ghost plane
 *     take the ghost value at every step; populations leaving are dropped);
 *   - PDFs are stored shifted, f_i - w_i rho0, in the storage precision;
 *     collision arithmetic is FP64 for PSM_FP64 storage and FP32 otherwise;
 *     force/torque sums are FP64;
 *   - the force/torque returned is the one ON THE BODY: minus the sums
 *     S_F = sum B sum_i Omega^S_i c_i and S_T = sum B (x - R) x sum_i Omega^S_i c_i
 *     of Eq. 10/11 (which are the momentum the solid gives the fluid).
 *
 * Pointers: every array argument may be a host pointer (pageable or pinned)
 * or a device pointer of the current device; the library copies with
 * cudaMemcpyDefault.  The library owns all device memory it allocates and
 * frees it in psm_destroy.  Calls on one handle are not thread safe.
 *
 * Errors: every function returns PSM_OK (0) or a negative PSM_ERR_* code and
 * records a message readable with psm_last_error() (thread local).  No C++
 * exception crosses the ABI and no kernel traps.
 */
#ifndef PSM_H_
#define PSM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSM_OK 0
#define PSM_ERR_ARG (-1)         /* invalid argument or configuration */
#define PSM_ERR_CUDA (-2)        /* a CUDA runtime call or a launch failed */
#define PSM_ERR_OOM (-3)         /* device or host allocation failed */
#define PSM_ERR_NONFINITE (-4)   /* a reduced result is NaN or infinite */
#define PSM_ERR_STATE (-5)       /* call out of order (e.g. backward before a recorded forward) */
#define PSM_ERR_UNSUPPORTED (-6) /* valid but not implemented combination */

#define PSM_MAX_BODIES 4

/* psm_lattice.stencil */
#define PSM_D3Q19 19
#define PSM_D3Q27 27
/* psm_lattice.streaming */
#define PSM_STREAM_AA 0       /* in place, one PDF copy (AA pattern, Sec. 2.2) */
#define PSM_STREAM_TWO_GRID 1 /* two PDF copies, push from the own cell */
/* psm_lattice.storage: PDF storage precision (values stored as f_i - w_i rho0) */
#define PSM_FP64 0
#define PSM_FP32 1
#define PSM_FP16_SHIFTED 2
#define PSM_BF16_SHIFTED 3
/* psm_collision.fluid */
#define PSM_BGK 0 /* single relaxation time, Eq. 2 */
#define PSM_TRT 1 /* two relaxation times: omega+ = 1/tau, Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) */
/* Cumulant operator (Geier et al. 2015; listed in the paper's Sec. 2.2, the
 * operator of every performance run in Sec. 5.1), D3Q19 only: central moments of the 19
 * exponent triples (a, b, c) in {0,1,2}^3 with at most two non-zero;
 * cumulants (order <= 3: the central moments; order 4:
 * C_220 = k_220 - (k_200 k_020 + 2 k_110^2) / rho and permutations) relaxed
 * towards rho c_s^2 delta (second order) and 0 (higher orders): the
 * off-diagonal and deviatoric second-order cumulants with 1/tau, their trace
 * with cum_omega[0], third order with cum_omega[1], fourth order with
 * cum_omega[2]; the PDFs are the unique D3Q19 set with the relaxed moments. */
#define PSM_CUMULANT 2
/* psm_collision.solid: SC1 (Eq. 7), SC2 (Eq. 8 as printed: u_s in both brackets), SC3 (Eq. 9) */
#define PSM_SC1 1
#define PSM_SC2 2
#define PSM_SC3 3
/* psm_collision.weighting */
#define PSM_B_DIRECT 0        /* B = eps, Eq. 5 */
#define PSM_B_TAU_WEIGHTED 1  /* B = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)), Eq. 6 */
/* psm_grid.bc_z */
#define PSM_BC_PERIODIC 0
#define PSM_BC_EQ_INLET_OUTLET 1

typedef struct psm_solver* psm_handle;

/* Grid: nx*ny*nz cells (each >= 1, nx*ny*nz < 2^32), rho0 > 0, |u_in| < 0.3. */
typedef struct {
  int64_t nx, ny, nz;
  int bc_z;          /* PSM_BC_PERIODIC or PSM_BC_EQ_INLET_OUTLET */
  double rho0;       /* reference density: storage shift and ghost-plane density */
  double u_in[3];    /* ghost-plane velocity */
} psm_grid;

typedef struct {
  int stencil;   /* PSM_D3Q19 or PSM_D3Q27 */
  int streaming; /* PSM_STREAM_AA or PSM_STREAM_TWO_GRID */
  int storage;   /* PSM_FP64, PSM_FP32, PSM_FP16_SHIFTED, PSM_BF16_SHIFTED */
} psm_lattice;

typedef struct {
  int fluid;          /* PSM_BGK, PSM_TRT or PSM_CUMULANT (D3Q19 only) */
  double tau;         /* relaxation time, > 1/2 (TRT: 1/omega+; cumulant: 1/shear rate) */
  double trt_lambda;  /* TRT Lambda (> 0); ignored otherwise.  3/16 is the usual choice */
  int solid;          /* PSM_SC1, PSM_SC2 or PSM_SC3 */
  int weighting;      /* PSM_B_DIRECT or PSM_B_TAU_WEIGHTED */
  double cum_omega[3]; /* PSM_CUMULANT: bulk, third-order and fourth-order rates, each in
                          (0, 2), or 0 for the default 1 (relax to equilibrium in one step);
                          ignored otherwise */
} psm_collision;

/*
 * Super-sampled binary geometry field of one body (Sec. 3), in the body frame.
 * The body-frame box [lo, lo + (gx, gy, gz)) is split into gx*gy*gz coarse
 * cells of size 1, each into (2^s)^3 sub-cells of size 2^-s (0 <= s <= 3).
 * A bit is 1 iff the sub-cell centre is inside the body.  Bits are packed per
 * coarse cell ("brick") into words_per_brick = max(1, 8^s / 64) 64-bit words:
 * bit b = (sz * 2^s + sy) * 2^s + sx of the brick, word b / 64, bit b % 64,
 * with (sx, sy, sz) the sub-cell offsets inside the coarse cell.  Bricks are
 * ordered [gz][gy][gx] (gx fastest).  bricks holds gx*gy*gz*words_per_brick
 * words.
 */
typedef struct {
  const uint64_t* bricks;
  int64_t gx, gy, gz;
  int s;
  double lo[3];
} psm_geom_field;

/* Synthetic rotor (hub cylinder plus twisted thin elliptic blades), body frame
 * with the hub axis along z:
 *   hub: sqrt(x^2 + y^2) <= r_hub and |z| <= hub_len / 2;
 *   blade k (0 <= k < n_blades) at azimuth phase + 2 pi k / n_blades, for
 *   r_hub <= r <= r_hub + span: with t = r * wrap(phi - azimuth) (wrap into
 *   [-pi, pi)), beta = hand * (pitch_root_deg - twist_deg (r - r_hub) / span)
 *   in radians, xi = t cos(beta) + z sin(beta), eta = -t sin(beta) + z cos(beta),
 *   inside iff (xi / (chord/2))^2 + (eta / (thickness/2))^2 <= 1. */
typedef struct {
  double r_hub, hub_len, span, chord, thickness, pitch_root_deg, twist_deg, phase;
  int n_blades;
  int hand; /* +1 or -1 */
} psm_rotor;

/* ------------------------------------------------------------------------ */
/* Library information                                                      */
/* ------------------------------------------------------------------------ */

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next call on this thread. */
const char* psm_last_error(void);

/* Lattice velocities (c_out: stencil*3 ints, may be NULL), weights (w_out:
 * stencil doubles, may be NULL) and opposite indices (opp_out, may be NULL)
 * in the library's direction order.  Host only; no GPU needed. */
int psm_lattice_velocities(int stencil, int* c_out, double* w_out, int* opp_out);

/* ------------------------------------------------------------------------ */
/* Geometry fields of analytic bodies (host helpers, no GPU needed)          */
/* ------------------------------------------------------------------------ */
/* Each voxeliser fills *out with a newly allocated host field (free it with
 * psm_geom_free).  Box rule: per axis, with e the body's half extent,
 * m = floor(e) + 2, lo = -m and 2m coarse cells, so sub-cell boundaries fall
 * on integers of the body frame.  Bits are set iff the sub-cell centre
 * satisfies the body's inside test (a point on the surface is inside). */

/* Sphere x^2 + y^2 + z^2 <= r^2. */
int psm_geom_voxelize_sphere(double r, int s, psm_geom_field* out);
/* Ellipsoid (x/a)^2 + (y/b)^2 + (z/c)^2 <= 1. */
int psm_geom_voxelize_ellipsoid(double a, double b, double c, int s, psm_geom_field* out);
/* Box |x| <= hx, |y| <= hy, |z| <= hz. */
int psm_geom_voxelize_box(double hx, double hy, double hz, int s, psm_geom_field* out);
/* Synthetic rotor (see psm_rotor). */
int psm_geom_voxelize_rotor(const psm_rotor* rotor, int s, psm_geom_field* out);
/* Closed triangle mesh (Sec. 3: the body's surface mesh is voxelised once
 * into this field), on the GPU.  vertices: nv x 3 floats (body frame, lattice
 * units), triangles: nt x 3 vertex indices, host or device.  A sub-cell is 1
 * iff a ray from its centre along +x crosses the surface an odd number of
 * times, decided exactly: the box is lo = floor(min v) - 1 to ceil(max v) + 1
 * per axis (at most 2^(19-s) cells), coordinates relative to lo are rounded
 * (half away from zero) to multiples of 2^-(s+8) cells, a centre on an edge or
 * vertex of the (y, z) projection counts as moved by (delta^2, delta) in
 * (y, z) for delta -> 0+, and a crossing at the centre's own x counts.  The
 * mesh must be closed (every edge shared by an even number of triangles) and
 * its components must not intersect; the result is host memory like the other
 * voxelisers'.  PSM_ERR_ARG: open mesh, bad index, degenerate index triple,
 * non-finite or too large coordinates; PSM_ERR_UNSUPPORTED: more than 256
 * crossings along one sub-cell row. */
int psm_geom_voxelize_mesh(const float* vertices, int64_t nv, const int32_t* triangles, int64_t nt, int s,
                           psm_geom_field* out);
/* Release a field returned by a voxeliser (bricks set to NULL). */
int psm_geom_free(psm_geom_field* field);

/* ------------------------------------------------------------------------ */
/* Solver                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a solver on the current CUDA device: the lattice of Sec. 2.2
 * (D3Q19 / D3Q27), the fluid collision Omega^F (BGK Eq. 2, TRT, or the
 * cumulant operator Sec. 2.2 / Sec. 5.1), the solid collision Omega^S
 * (Eq. 7/8/9) and the weighting B (Eq. 5 / Eq. 6) of the PSM update Eq. 4,
 * and the inflow of Sec. 5.1's flow set-ups.  stream: a cudaStream_t (NULL =
 * the legacy default stream) on which every kernel of this handle runs.
 * Validates tau > 1/2, |u_in| < 0.3, rho0 > 0, trt_lambda > 0, the grid size
 * and the enum values (PSM_ERR_ARG), allocates the PDF buffer(s) and the
 * reduction scratch (PSM_ERR_OOM).  The PDFs are initialised to the
 * equilibrium f^eq(rho0, u_in).  The step counter starts at 0. */
int psm_create(const psm_grid* grid, const psm_lattice* lattice, const psm_collision* collision, void* stream,
               psm_handle* out);

/* psm_create on caller-owned PDF buffers (for instance PyTorch tensors):
 * buffers[0] (and buffers[1] for two-grid streaming) are device pointers to
 * Q * nx * ny * nz elements of the storage type each (shifted f - w rho0,
 * natural layout [Q][nz][ny][nx] in the library's direction order), 16-byte
 * aligned, distinct.  The caller keeps ownership: psm_destroy never frees
 * them and they must outlive the handle.  flags: 0 initialises the state to
 * f^eq(rho0, u_in) like psm_create; PSM_BUFFERS_KEEP keeps buffers[0]'s
 * contents as the state at step 0.  PSM_ERR_ARG for NULL, misaligned or equal
 * buffers or unknown flags (before any CUDA call), and for a buffer that is
 * not device memory of the current device (or managed memory) or whose
 * allocation ends before Q * ncell elements (checked with
 * cudaPointerGetAttributes and the driver's address range, before any
 * launch: a host pointer would fault the kernels). */
#define PSM_BUFFERS_KEEP 1
int psm_create_with_buffers(const psm_grid* grid, const psm_lattice* lattice, const psm_collision* collision,
                            void* stream, void* const* buffers, int flags, psm_handle* out);

/* Free everything the handle owns.  NULL is accepted. */
int psm_destroy(psm_handle h);

/* Set every cell to f^eq(rho, u) (Eq. 3), keeping the step counter; populations
 * entering from a z ghost plane take the ghost value. */
int psm_init_equilibrium(psm_handle h, double rho, const double u[3]);

/* The same from per-cell fields: rho[nz][ny][nx] (> 0) and u[nz][ny][nx][3]
 * (|u| < 0.3), host or device, FP64 (PSM_ERR_ARG naming the first bad cell). */
int psm_init_equilibrium_field(psm_handle h, const double* rho, const double* u);

/* Import / export the full PDF state, natural layout, FP64, unshifted f,
 * [Q][nz][ny][nx] in the library's direction order (Q*nx*ny*nz doubles).
 * Import rounds to the storage precision.  Export of a state in the AA
 * "swapped" layout (after an odd number of AA steps) undoes the swap. */
int psm_set_state(psm_handle h, const double* f);
int psm_get_state(psm_handle h, double* f);

/* The stored PDFs in the storage precision: shifted f - w rho0, natural
 * layout [Q][nz][ny][nx] (un-swapped after an odd AA step; populations
 * entering from a z ghost plane as the ghost value), Q * ncell elements of
 * the storage type, host or device. */
int psm_get_pdfs(psm_handle h, void* f);

/* Natural, unshifted FP64 PDFs of n listed cells (flat indices
 * (z * ny + y) * nx + x, host or device): f[n][Q] in the library's direction
 * order.  PSM_ERR_ARG for an index out of range.  For sampled checks of grids
 * too large to export whole. */
int psm_get_cells(psm_handle h, const int64_t* cells, int64_t n, double* f);

/* Density and velocity u = j / rho per cell: rho[nz][ny][nx], u[nz][ny][nx][3] (FP64). */
int psm_get_macroscopic(psm_handle h, double* rho, double* u);

/* Solid fraction eps (Sec. 3, all bodies combined: min(1, sum_b eps_b)) at the
 * pose of the current step counter: eps[nz][ny][nx] (float; exact multiples
 * of 2^-3s). */
int psm_get_eps(psm_handle h, float* eps);

/* Attach body `body` (0 <= body < PSM_MAX_BODIES; bodies are used in id order
 * and must be set contiguously from 0): the super-sampled binary geometry
 * field of Sec. 3, voxelised once and copied to the device once; every step
 * maps it onto eps through the body's pose (Sec. 3: the cell centre rotated
 * into the body frame and translated).  Motion: pose at step n is Q_n = Rot(omega/|omega|, |omega| n) Q0
 * (Rodrigues), R_n = R0 + v n; Q0 is row-major world <- body; R0 is the
 * reference point (centre of rotation, torque reference).  Solid velocity
 * u_s(x) = omega x (x - R_n) + v.  Replacing a body is allowed. */
int psm_set_geometry(psm_handle h, int body, const psm_geom_field* field, const double Q0[9], const double R0[3],
                     const double omega[3], const double v[3]);

/* Angular velocity of body `body` in its solid velocity u_s = omega x (x - R_n)
 * + v (Eq. 7-9) from the next step on, while its pose sequence (Sec. 3) keeps
 * the omega of psm_set_geometry: the geometry stays frozen when u_s's omega
 * changes, which is how psm_backward differentiates with respect to omega
 * (central differences of J in this omega check grad_omega).
 * psm_set_geometry resets it to the pose's omega.  PSM_ERR_ARG for a bad body
 * or non-finite values; PSM_ERR_STATE for a two-way coupled body. */
int psm_set_us_omega(psm_handle h, int body, const double omega[3]);

/* Number of bodies attached. */
int psm_num_bodies(psm_handle h, int* out);

/* Two-way coupling (the paper's validation with a freely settling sphere,
 * Sec. 4; the performance runs couple one way).  From the current step on,
 * body `body` moves under the force and torque the fluid exerts on it (the
 * values psm_force_torque returns) plus constant external loads, one
 * semi-implicit Euler step of the rigid-body equations per time step (dt = 1):
 *   v += (F + force_ext) / mass,  R += v,  L += T + torque_ext,
 *   Q <- Rot(w*) Q  with w* = Q I^-1 Q^T L,  then w = Q I^-1 Q^T L,
 * integrated on the device in FP64 after each step (no host synchronisation).
 * The state starts from the prescribed motion at the current step (R_n, Q_n,
 * v, omega, L = Q I Q^T omega); R is the torque reference point and should be
 * the centre of mass.  Explicit coupling needs the body heavier than the fluid
 * it displaces (otherwise the added-mass instability).  psm_set_geometry on
 * the body returns it to prescribed motion.  PSM_ERR_ARG for a bad body, a
 * non-positive mass or an inertia that is not symmetric positive definite;
 * PSM_ERR_STATE while recording for psm_backward (which supports prescribed
 * motion only) or with the remap frozen. */
typedef struct {
  double mass;          /* > 0 (lattice units: fluid density rho0 per cell) */
  double inertia[9];    /* body-frame inertia about R, row-major, symmetric positive definite */
  double force_ext[3];  /* constant external force, world frame (e.g. gravity minus buoyancy) */
  double torque_ext[3]; /* constant external torque about R, world frame */
} psm_body_dynamics;
int psm_set_body_dynamics(psm_handle h, int body, const psm_body_dynamics* dyn);

/* Motion of body `body` for the next step to run: R[3], v[3], Q[9]
 * (world <- body, row-major), omega[3], L[3] (21 doubles; L = 0 for prescribed
 * motion).  Synchronises. */
int psm_body_state(psm_handle h, int body, double* out);

/* Remapping of the moving geometry onto eps (Sec. 3): every_step = 1
 * (default) remaps at every step from that step's pose; 0 freezes the poses of
 * all bodies at the current step (eps, the reference point R and the lever
 * arm of u_s stay those of that step; omega and v still give u_s), as for a
 * body whose geometry is static.  PSM_ERR_STATE while recording. */
int psm_set_remap(psm_handle h, int every_step);

/* Run n >= 0 time steps asynchronously on the handle's stream (one fused
 * kernel launch per step; no host synchronisation).  One step is the pose and
 * remap of Sec. 3, the PSM collision Eq. 4 (with Eq. 2/3, Eq. 5/6, Eq. 7-9),
 * streaming Eq. 1 and the force/torque sums Eq. 10/11, in that order. */
int psm_step(psm_handle h, int n);

/* Step counter (steps taken since creation). */
int psm_step_count(psm_handle h, int64_t* out);

/* Force (3) and torque (3) on body `body` for steps [step_from, step_from +
 * count): out[count][6] (FP64), the negatives of Eq. 10 / Eq. 11 (the sums
 * over the cells the body owns with B > 0, torque about R_n).  Synchronises the stream.  Only the last
 * psm_series_capacity() steps are kept (PSM_ERR_ARG for older steps).
 * PSM_ERR_NONFINITE if any returned value is NaN or infinite. */
int psm_force_torque(psm_handle h, int body, int64_t step_from, int64_t count, double* out);
/* The same series with the sign of Eq. 10 / 11 as printed (the momentum the
 * solid gives the fluid): the negative of psm_force_torque. */
int psm_force_torque_raw(psm_handle h, int body, int64_t step_from, int64_t count, double* out);
int psm_series_capacity(psm_handle h, int64_t* out);

/* Total mass sum_x sum_i f_i (FP64, deterministic order).  Synchronises.
 * PSM_ERR_NONFINITE if it is not finite. */
int psm_mass(psm_handle h, double* out);

/* Wait for all work of the handle.  PSM_ERR_CUDA if a step kernel gave up
 * waiting for its staged loads, or refused a tiling it was not built for (it
 * records this in a flag instead of trapping). */
int psm_synchronize(psm_handle h);

/* Step-kernel variant: PSM_KERNEL_AUTO (default) uses the TMA-staged kernel
 * for every step the shape allows (the faster variant measured on GB300), else
 * plain global loads;
 * PSM_KERNEL_PLAIN forces plain loads; PSM_KERNEL_TMA forces TMA staging for
 * every step the shape allows (PSM_ERR_UNSUPPORTED if it allows none).  TMA
 * shapes: with TX = min(256, nx): nx % TX == 0, 256 % nx == 0 when nx < 256,
 * TX >= 32, ny % (256 / TX) == 0 (ny % (512 / TX) == 0 for the D3Q19
 * two-grid BGK/TRT step in FP16/BF16, whose tiles hold two cells per thread),
 * nx * sizeof(PDF) a multiple of 16 bytes, staging buffers within the
 * per-block shared memory; the AA odd step also needs TX = 256.  All variants
 * compute the same states, bit for bit; the FP64 force/torque sums agree bit
 * for bit where the variants tile alike and to rounding (summation order)
 * otherwise. */
/* ------------------------------------------------------------------------ */
/* z-slab decomposition (Sec. 5.2 runs one block of the lattice per GPU and    */
/* exchanges the populations that cross block faces every step)              */
/* ------------------------------------------------------------------------ */

/* Declare the handle's lattice the planes [z0, z0 + nz) of a larger domain:
 * cell centres (the remap, u_s, the torque lever arm) use the world z + z0;
 * force, torque and mass are then this slab's part of the sums (add them over
 * the slabs).  A slab is created with bc_z = PSM_BC_PERIODIC: the periodic
 * wrap puts the populations that leave through one face into the slots of the
 * opposite face, from where the caller's exchange moves them to the
 * neighbouring slab between steps (psm_slot_plane; after every two-grid step,
 * before and after every odd AA step), or replaces them with the inflow
 * equilibrium at the domain's own z ends (psm_fill_slot_plane).  PSM_ERR_ARG
 * for z0 < 0 or z0 + nz > 2^30; PSM_ERR_STATE while recording or with
 * two-way coupled bodies; afterwards psm_record and psm_set_body_dynamics
 * refuse the handle (the adjoint and the free-body update are not
 * decomposed). */
int psm_set_z_offset(psm_handle h, int64_t z0);

/* Device address of slot `slot` (0 <= slot < Q, the library's direction
 * order) of plane z (0 <= z < nz) in the buffer the next step reads: nx * ny
 * contiguous values of the storage type, stored as the step kernels keep them
 * (shifted; the AA pattern's swapped layout after an odd step).  Valid until
 * the next psm_step (two-grid streaming alternates buffers); for the face
 * exchange of a slab decomposition (a peer copy or NCCL send/recv into each
 * GPU's own buffers). */
int psm_slot_plane(psm_handle h, int slot, int z, void** out);

/* Set slot `slot` of plane z, in the buffer the next step reads, to the
 * inflow equilibrium f^eq_dir(rho0, u_in) of direction `dir` held by the
 * ghost planes (shifted, rounded to the storage type), asynchronously on the
 * handle's stream.  dir = slot in the natural layout; in the AA pattern's
 * swapped layout slot opp(i) holds population i, so dir = opp(slot).  Used at
 * the ends of a decomposed domain whose z is bounded by ghost planes. */
int psm_fill_slot_plane(psm_handle h, int slot, int z, int dir);

/* ------------------------------------------------------------------------ */
/* Differentiation (not in the paper): discrete adjoint of the step          */
/* ------------------------------------------------------------------------ */

/* Per-cell additive perturbation delta of the solid fraction: every step uses
 * B(eps_n(x) + delta(x)) (Eq. 5 / 6, not clamped).  delta: ncell floats
 * [nz][ny][nx], host or device, copied; NULL removes it. */
int psm_set_eps_delta(psm_handle h, const float* delta);

/* Start recording the trajectory for psm_backward at the current step n0 (the
 * forward map recorded is the step of psm_step: Sec. 3, Eq. 1-11):
 * the state is checkpointed now and before every K-th later step (device
 * memory, stream-ordered allocation), and the buffers of psm_backward are
 * allocated.  K = 0 stops recording and frees the checkpoints.  With AA
 * streaming, n0 and K must be even.  flags:
 * PSM_RECORD_INIT_FROM_INFLOW declares that the state at n0 is
 * f^eq(rho0, u_in) (psm_create or psm_init_equilibrium(rho0, u_in)), so that
 * the gradient with respect to u_in includes the initial state.
 * PSM_RECORD_SEQUENTIAL keeps psm_backward to one set of recompute buffers
 * (no second set, see psm_backward; a set allocated before is freed).
 * PSM_ERR_UNSUPPORTED for the cumulant operator (the adjoint step is written
 * for BGK and TRT). */
#define PSM_RECORD_INIT_FROM_INFLOW 1
#define PSM_RECORD_SEQUENTIAL 2
int psm_record(psm_handle h, int K, int flags);

/* Gradient of J = sum_{n, body, k} w[n][body][k] * FT[n][body][k] over the
 * recorded steps n0 <= n < step (FT as psm_force_torque returns it) by the
 * discrete adjoint: segments between checkpoints are recomputed (two-grid
 * step kernel) and swept backwards with the adjoint step kernel.
 *   dJ_dFT:     w, (step - n0) * nbodies * 6 doubles; NULL = mean torque
 *               about z on body 0, w[n][0][5] = 1 / (step - n0);
 *   grad_eps:   dJ/d delta per cell, ncell doubles (NULL: not returned);
 *   grad_omega: dJ/d omega per body (the geometry sequence is held fixed:
 *               omega enters through u_s only), nbodies * 3 doubles (or NULL);
 *   grad_uin:   dJ/d u_in (ghost planes, plus the initial state if recorded
 *               with PSM_RECORD_INIT_FROM_INFLOW), 3 doubles (or NULL).
 * Adjoint arithmetic is FP32 (FP64 for PSM_FP64 storage); sums are FP64.
 * Its buffers (K - 1 recompute states, two adjoint fields, the FP64
 * gradient) are allocated by psm_record and kept by the handle until
 * psm_destroy or a recording with another K.  Where a second set of K - 1
 * states fits with a sixteenth of the device memory left free, psm_record
 * allocates it too, with a stream of the handle's own: psm_backward then
 * recomputes the segment before the current one on that stream while the
 * adjoint sweeps the current one (same results, bit for bit).
 * Synchronises; the handle keeps its state and step counter.
 * PSM_ERR_STATE without a recorded forward. */
int psm_backward(psm_handle h, const double* dJ_dFT, double* grad_eps, double* grad_omega, double* grad_uin);

/* ------------------------------------------------------------------------ */
/* Allocation-free reduction (no counterpart in the paper)                   */
/* ------------------------------------------------------------------------ */

/* Total mass sum_x sum_i f_i of a caller-owned PDF field, for callers that
 * must not allocate device memory (an application that routes every device
 * allocation through its own pool, or a loop that cannot afford the implicit
 * device synchronisation of cudaMalloc).  It allocates nothing: its scratch
 * (block partial sums, a ticket counter, the result) is a file-scope
 * __device__ array of about 128 KB that every GPU loading the library holds
 * until the process exits.
 *   f:       device pointer, [Q][ncell] values in the storage precision
 *            `storage` (PSM_FP64 ... PSM_BF16_SHIFTED), stored as
 *            f_i - w_i rho0 (pass rho0 = 0 for unshifted values);
 *   stencil: PSM_D3Q19 or PSM_D3Q27;  ncell: 1 .. 2^30 (PSM_ERR_ARG beyond:
 *            the scratch holds 16384 partial sums of 65536 cells each);
 *   stream:  cudaStream_t (NULL = legacy default stream);
 *   out:     one double, host or device.
 * The call synchronises `stream` before it returns (it reads the result back
 * to the host to test it).  PSM_ERR_ARG if f is not device memory of the
 * current device (or managed memory) holding Q * ncell values (checked before
 * the launch).  The summation order is fixed (deterministic).  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) for
 * that device and keeps it for the life of the process (do not use the
 * function across a cudaDeviceReset).  All calls share the one array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller. */
int psm_mass_noalloc(const void* f, int storage, int stencil, int64_t ncell, double rho0, void* stream,
                     double* out);

/* Host-side check of a caller-owned buffer (no counterpart in the paper; the
 * check psm_create_with_buffers and psm_mass_noalloc make): PSM_OK when p
 * points into device memory of the current device, or managed memory, and
 * its allocation holds at least `bytes` bytes from p on (where the driver
 * reports the allocation's extent); PSM_ERR_ARG otherwise, with the reason in
 * psm_last_error() (host memory, another device's memory, too small).
 * Launches nothing and allocates nothing. */
int psm_check_device_buffer(const void* p, int64_t bytes);

#define PSM_KERNEL_AUTO 0
#define PSM_KERNEL_PLAIN 1
#define PSM_KERNEL_TMA 2
int psm_set_kernel_variant(psm_handle h, int variant);
/* The variant psm_step uses now (PSM_KERNEL_PLAIN or PSM_KERNEL_TMA). */
int psm_kernel_variant(psm_handle h, int* out);

/* Diagnostics (host only, no GPU needed): the shared-memory layout the
 * TMA-staged step kernel is built with for `storage`, `stencil`, `mode`
 * (0 two-grid, 1 AA even step, 2 AA odd step) and `fluid`:
 *   out[0] dynamic shared memory per block (bytes), out[1] pipeline stages,
 *   out[2] resident blocks per SM it is sized for, out[3] cells per thread.
 * The stages fill 228 KB per SM over out[2] blocks, less 1 KB reserved and
 * 6 KB of static shared memory per block.  PSM_ERR_ARG for an unknown value,
 * PSM_ERR_UNSUPPORTED for the cumulant operator on D3Q27. */
int psm_tma_layout(int storage, int stencil, int mode, int fluid, int* out);

#ifdef __cplusplus
}
#endif

#endif /* PSM_H_ */
