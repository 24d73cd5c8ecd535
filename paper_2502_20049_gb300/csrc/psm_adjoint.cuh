// Discrete adjoint (reverse-time) PSM step.  Not in the paper: it is the exact
// transpose of the forward step of psm_kernels.cuh, for gradients of a linear
// functional J of the force/torque series with respect to a per-cell
// perturbation delta of the solid fraction, the angular velocities and the
// inflow velocity.
//
// Forward step n (pre-collision state f^n, natural layout):
//   f^{n+1} = S(C_n(f^n)),   C_n = per-cell Eq. 4 with B = B(eps_n + delta),
//   S = streaming (pull from x - c_i; ghost value where x - c_i is outside).
// Adjoint step n, per cell y, with mu_i(y) = lambda^{n+1}_i(y + c_i) (zero where
// y + c_i is outside: the population left the domain):
//   lambda^n(y) = (dC_n/df)^T mu(y) + dJ_n/df(y),
//   dJ/d delta(y) += [mu . dC_n/dB + dJ_n/dB] B'(eps + delta),
//   dJ/d omega_b  += (x_c - R_n) x (dJ/du_s) over the cells owned by body b,
//   dJ/d u_in     += lambda^n_i(y) d g_i/d u_in for populations taken from a
//                    ghost plane (g_i = f^eq_i(rho0, u_in)).
// The eps sequence is the forward's (frozen geometry: eps is piecewise
// constant in omega).  All arithmetic is in the compute precision T (FP32 for
// FP32/FP16/BF16 storage, FP64 for FP64), the per-cell terms of the scalar
// gradients and their 32-cell warp partials included (on GB300 an FP64
// instruction costs about 64 FP32 ones); the warp partials are added into FP64
// block slots and summed in FP64 in a fixed order.
#pragma once

#include "psm_kernels.cuh"

namespace psm {

struct AdjParams {
  Grid3 g;
  Tiling t;
  const void* f;        // f^n, natural layout, storage S, shifted
  const void* lam_in;   // lambda^{n+1}, [Q][ncell] in T
  void* lam_out;        // lambda^n
  double* grad;         // [ncell]: += dJ/d delta (FP64 accumulator)
  int trt, solid, weighting, nbodies;
  DevBody body[PSM_MAX_BODIES];
  const float* delta;
  const double* w;      // [nbodies][6] weights of this step's force/torque in J (null: none)
  double dghost[27][3]; // d g_i / d u_in
  float dghostf[27][3]; // the same in FP32
  double* partials;
  unsigned int* ticket;
  double* acc_out;      // [nbodies * 3 + 3]: dJ/d omega per body, dJ/d u_in
  ConstT<float> cf;
  ConstT<double> cd;
  // slot base pointers (elements): f + i ncell (storage S), lam_in / lam_out + i ncell (T)
  const void* f_slot[27];
  const void* lin_slot[27];
  void* lout_slot[27];
};

#define PSM_DECLARE_ADJOINT(NAME)                                                              \
  cudaError_t launch_adjoint_##NAME(int Q, int trt, const AdjParams& p, cudaStream_t st);      \
  cudaError_t launch_adjoint_init_##NAME(int Q, const AdjParams& p, int blocks, cudaStream_t st);
PSM_DECLARE_ADJOINT(fp64)
PSM_DECLARE_ADJOINT(fp32)
PSM_DECLARE_ADJOINT(fp16)
PSM_DECLARE_ADJOINT(bf16)

template <class T>
__device__ __forceinline__ const ConstT<T>& acst(const AdjParams& p) {
  if constexpr (sizeof(T) == 4) return p.cf;
  else return p.cd;
}

// phi_i(v) = d f^eq_i / d rho = w_i (1 + 3 c.v + 4.5 (c.v)^2 - 1.5 v.v)
template <int Q, class T>
__device__ __forceinline__ T phi(int i, T cv, T vv) {
  return T(lat_w<Q>(i)) * (T(1) + T(3) * cv + T(4.5) * cv * cv - T(1.5) * vv);
}

// Adjoint of one cell whose forward is the pure fluid collision (B = 0: no
// body box and no eps perturbation in its tile, so u_s = 0 and nothing of the
// force/torque) with no ghost population.  mu_i = lambda^{n+1}_i(x + c_i).
// Writes lambda^n(x) to lam and returns mu . d post / d B (the factor of
// B'(eps) in dJ/d delta).  The forward per opposite pair (fluid_relax):
//   p = (1 - w+) s/2 + w+ even,  m = (1 - w-) d/2 + w- odd,  f*_i = p + m, f*_j = p - m,
//   even = w (base + 4.5 rho cu^2), odd = 3 w rho cu,  base = drho - 1.5 rho u.u;
// reversed with pb = mu_i + mu_j, mb = mu_i - mu_j:
//   fbar_i = (1 - w+)/2 pb + (1 - w-)/2 mb,  fbar_j = (1 - w+)/2 pb - (1 - w-)/2 mb,
//   basebar += w w+ pb,  rhobar += cu (4.5 w w+ cu pb + 3 w w- mb),
//   ubar += rho c (9 w w+ cu pb + 3 w w- mb),
// then through base, u = j / rho and the moments.  The B-derivative
// mu . (Omega^S - Omega^F) per pair, with G = w drho (f^eq at u_s = 0) and
// mu . Omega^F = w+ pb (even - s/2) + w- mb (odd - d/2):
//   SC1: mu . Omega^S = (G - even) pb + (odd - d) mb
//   SC2: mu . Omega^S = (G pb - (pb s + mb d)/2) / tau
//   SC3: mu . Omega^S = -d mb
template <class T, int Q>
__device__ __forceinline__ T adj_fluid_cell(const ConstT<T>& C, int solid, T inv_tau, const T (&f)[Q],
                                            const T (&mu)[Q], T (&lam)[Q]) {
  const T omp = C.om_a + C.om_b, omm = C.om_a - C.om_b;
  T drho, rho, ux, uy, uz, uu;
  moments<T, Q>(f, C.rho0, drho, rho, ux, uy, uz, uu);
  const T inv_rho = recip(rho);
  const T base = drho - T(1.5) * rho * uu;
  // rest population: f*_0 = (1 - w+) f_0 + w+ w_0 base
  T baseb = C.pw[0] * mu[0];
  lam[0] = C.omp1 * mu[0];
  T bb;
  {
    const T w0 = T(lat_w<Q>(0));
    const T n0 = f[0] - w0 * base, m0 = f[0] - w0 * drho;
    const T os0 = solid == PSM_SC1 ? n0 - m0 : (solid == PSM_SC2 ? -m0 * inv_tau : T(0));
    bb = mu[0] * (os0 + omp * n0);
  }
  T rhob = T(0), upx = T(0), upy = T(0), upz = T(0);  // upx..: u adjoint along c, without the factor rho
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int j = i + 1, c = lat_cls(i);
    const T w = T(lat_w<Q>(i));
    const T cu = cdot(i, ux, uy, uz);
    const T sp = f[i] + f[j], dm = f[i] - f[j];
    const T pb = mu[i] + mu[j], mb = mu[i] - mu[j];
    const T a1 = C.pk[c] * cu;
    const T t = a1 * pb + C.pd[c] * mb;
    rhob += cu * t;
    const T t2 = a1 * pb + t;
    if (lat_cx(i)) upx += csign(lat_cx(i), t2);
    if (lat_cy(i)) upy += csign(lat_cy(i), t2);
    if (lat_cz(i)) upz += csign(lat_cz(i), t2);
    baseb += C.pw[c] * pb;
    const T hm = C.hm1 * mb;
    lam[i] = C.hp1 * pb + hm;
    lam[j] = C.hp1 * pb - hm;
    // mu . (Omega^S - Omega^F) of the pair
    const T wr = w * rho;
    const T even = w * base + T(4.5) * wr * (cu * cu), odd = T(3) * wr * cu;
    const T muof = omp * pb * (even - T(0.5) * sp) + omm * mb * (odd - T(0.5) * dm);
    T muos;
    if (solid == PSM_SC1) muos = (w * drho - even) * pb + (odd - dm) * mb;
    else if (solid == PSM_SC2) muos = (w * drho * pb - T(0.5) * (pb * sp + mb * dm)) * inv_tau;
    else muos = -dm * mb;
    bb += muos - muof;
  }
  // base = drho - 1.5 rho u.u
  T drhob = baseb;
  rhob += T(-1.5) * uu * baseb;
  const T uub = T(-1.5) * rho * baseb;
  // u.u, then u = j / rho
  const T ubx = rho * upx + T(2) * ux * uub, uby = rho * upy + T(2) * uy * uub, ubz = rho * upz + T(2) * uz * uub;
  const T jbx = ubx * inv_rho, jby = uby * inv_rho, jbz = ubz * inv_rho;
  rhob -= (ubx * ux + uby * uy + ubz * uz) * inv_rho;
  drhob += rhob;  // rho = rho0 + drho
#pragma unroll
  for (int i = 0; i < Q; ++i) lam[i] += drhob + cdot(i, jbx, jby, jbz);
  return bb;
}

// PART: 0 every tile; 1 the fluid-only tiles (no scalar sums: a lean kernel
// that fits three blocks per SM); 2 the general tiles (with the FP64 sums).
// A step launches 1 and 2 (disjoint cells) or 0.
template <class S, int Q, int TRT, int PART>
__global__ void __launch_bounds__(PSM_THREADS, sizeof(S) == 8 ? 1 : (PART == 1 ? 3 : 2))
    k_adjoint(const __grid_constant__ AdjParams p) {
  using T = typename Store<S>::T;
  constexpr int NW = PSM_THREADS / 32;
  constexpr int NC = PSM_MAX_BODIES * 3 + 3;
  __shared__ double s_acc[NW][NC];
  const int nb = p.nbodies;
  const int ncomp = nb * 3 + 3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = lane; k < NC; k += 32) s_acc[warp][k] = 0.0;
  double* __restrict__ grad = p.grad;
  const ConstT<T>& C = acst<T>(p);
  const T om_a = C.om_a, om_b = C.om_b, inv_tau = C.inv_tau;
  const int ntiles = (int)p.t.ntiles;
  const int lx = (int)threadIdx.x % p.t.tx, ly = (int)threadIdx.x / p.t.tx;
  // B'(0): the derivative of the weighting at eps = 0 (fluid-only tiles)
  const T Bp0 = p.weighting == PSM_B_TAU_WEIGHTED ? C.tmh / (T(1) + C.tmh) : T(1);

  // One cell.  GEN: the tile meets a body's cell box, a ghost plane, or an eps
  // perturbation is set; the other tiles' cells take adj_fluid_cell.
  auto cell_body = [&](auto gen_c, int x, int y, int z) {
    constexpr bool GEN = decltype(gen_c)::value;
    const bool active = x < p.g.nx && y < p.g.ny;
    T aw0 = 0, aw1 = 0, aw2 = 0, au0 = 0, au1 = 0, au2 = 0;
    bool has_w = false, has_u = false;
    int owner = -1;
    if (active) {
      const unsigned cell = ((unsigned)z * (unsigned)p.g.ny + (unsigned)y) * (unsigned)p.g.nx + (unsigned)x;
      Stencil sn;
      sn.init(p.g, x, y, z, cell);
      ZGhost zg;
      zg.init(p.g, z);
      // the gradient accumulator is read with the PDFs and the adjoint field, so
      // that its read-modify-write at the end does not add a second memory round
      // trip (each cell belongs to one thread of the launch)
      const double g_old = grad[cell];
      T f[Q], mu[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int cx = lat_cx(i), cy = lat_cy(i), cz = lat_cz(i);
        if (GEN && zg.from(cz)) f[i] = C.ghost[i];
        else f[i] = Store<S>::ld(static_cast<const S*>(p.f_slot[i]) + cell);
        mu[i] = (GEN && zg.to(cz)) ? T(0) : static_cast<const T*>(p.lin_slot[i])[sn.at(cx, cy, cz)];
      }
      if constexpr (!GEN) {
        T lam[Q];
        const T bb = adj_fluid_cell<T, Q>(C, p.solid, inv_tau, f, mu, lam);
#pragma unroll
        for (int i = 0; i < Q; ++i) static_cast<T*>(p.lout_slot[i])[cell] = lam[i];
        grad[cell] = g_old + (double)(bb * Bp0);
      } else {
      // ---- forward recomputation (same arithmetic as psm_collide) ----
      float epsf = 0.0f;
      if (GEN) epsf = cell_eps(p.body, nb, x, y, z, owner);
      T e = T(epsf);
      if (p.delta) e += T(p.delta[cell]);
      if (e == T(0)) {
        // B = 0 (a cell of a general tile outside the bodies): the fluid-only
        // reverse step, B'(0) for the gradient.  On a ghost plane the
        // populations entering from it hold the ghost values g_i(u_in) (loaded
        // so above, mu = 0 for those leaving into it), and their adjoint adds
        // to dJ/d u_in.
        T lam[Q];
        const T bb = adj_fluid_cell<T, Q>(C, p.solid, inv_tau, f, mu, lam);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          static_cast<T*>(p.lout_slot[i])[cell] = lam[i];
          if (zg.from(lat_cz(i))) {
            if constexpr (sizeof(T) == 4) {
              au0 += lam[i] * p.dghostf[i][0];
              au1 += lam[i] * p.dghostf[i][1];
              au2 += lam[i] * p.dghostf[i][2];
            } else {
              au0 += lam[i] * p.dghost[i][0];
              au1 += lam[i] * p.dghost[i][1];
              au2 += lam[i] * p.dghost[i][2];
            }
            has_u = true;
          }
        }
        grad[cell] = g_old + (double)(bb * Bp0);
      } else {
        T Bw = e, Bp = T(1);
        if (p.weighting == PSM_B_TAU_WEIGHTED) {
          const T t = C.tmh;
          const T den = (T(1) - e) + t;
          Bw = e * t / den;
          Bp = t * (T(1) + t) / (den * den);
        }
        T drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          drho += f[i];
          if (lat_cx(i)) jx += T(lat_cx(i)) * f[i];
          if (lat_cy(i)) jy += T(lat_cy(i)) * f[i];
          if (lat_cz(i)) jz += T(lat_cz(i)) * f[i];
        }
        const T rho = C.rho0 + drho;
        const T inv_rho = recip(rho);
        const T ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
        const T uu = ux * ux + uy * uy + uz * uz;
        T usx = 0, usy = 0, usz = 0;
        T Rx = 0, Ry = 0, Rz = 0;
        if (GEN && owner >= 0) {
          const DevBody& b = p.body[owner];
          T rx, ry, rz, wx, wy, wz, vx, vy, vz;
          if constexpr (sizeof(T) == 4) {
            rx = (T(x) + T(0.5)) - b.Rf[0];
            ry = (T(y) + T(0.5)) - b.Rf[1];
            rz = (T(z) + T(0.5)) - b.Rf[2];
            wx = b.omegaf[0], wy = b.omegaf[1], wz = b.omegaf[2];
            vx = b.vf[0], vy = b.vf[1], vz = b.vf[2];
          } else {
            rx = (double)x + 0.5 - b.R[0];
            ry = (double)y + 0.5 - b.R[1];
            rz = (double)z + 0.5 - b.R[2];
            wx = b.omega[0], wy = b.omega[1], wz = b.omega[2];
            vx = b.v[0], vy = b.v[1], vz = b.v[2];
          }
          Rx = rx, Ry = ry, Rz = rz;
          usx = wy * rz - wz * ry + vx;
          usy = wz * rx - wx * rz + vy;
          usz = wx * ry - wy * rx + vz;
        }
        const T usus = usx * usx + usy * usy + usz * usz;
        const T omB = T(1) - Bw;
        // ---- adjoint of the force/torque terms: s = B sum_i Omega^S_i c_i ----
        T sbx = 0, sby = 0, sbz = 0;
        if (GEN && owner >= 0 && Bw > T(0) && p.w) {
          const double* wv = p.w + owner * 6;
          // J_n = sum_b w_F . F_b + w_T . T_b with F_b = -sum s, T_b = -sum r x s
          const T w0 = T(wv[0]), w1 = T(wv[1]), w2 = T(wv[2]), w3 = T(wv[3]), w4 = T(wv[4]), w5 = T(wv[5]);
          sbx = -(w0 + (w4 * Rz - w5 * Ry));
          sby = -(w1 + (w5 * Rx - w3 * Rz));
          sbz = -(w2 + (w3 * Ry - w4 * Rx));
        }
        // ---- reverse sweep over the rest population and the opposite pairs ----
        T Bbar = 0, rhob = 0;
        T ubx = 0, uby = 0, ubz = 0, usbx = 0, usby = 0, usbz = 0;
        // Without an owner (the fast path), u_s = 0: G_i = f^eq_i(rho, 0) - w_i rho0
        // = w_i drho, phi_i(0) = w_i, and there is no u_s adjoint to accumulate.
        {
          const T E0 = feq_shifted_nz<Q, T>(0, drho, rho, ux, uy, uz, uu);
          const T G0 = GEN ? feq_shifted_nz<Q, T>(0, drho, rho, usx, usy, usz, usus) : T(lat_w<Q>(0)) * drho;
          const T n0 = f[0] - E0, m0 = f[0] - G0;
          const T of0 = -(om_a + om_b) * n0;
          T os0;
          if (p.solid == PSM_SC1) os0 = n0 - m0;
          else if (p.solid == PSM_SC2) os0 = -m0 * inv_tau;
          else os0 = T(0);
          const T osb = Bw * mu[0], ofb = omB * mu[0];
          Bbar += mu[0] * (os0 - of0);
          T nb0 = -(om_a + om_b) * ofb, mb0;
          if (p.solid == PSM_SC1) {
            nb0 += osb;
            mb0 = -osb;
          } else if (p.solid == PSM_SC2) {
            mb0 = -osb * inv_tau;
          } else {
            mb0 = T(0);
          }
          f[0] = mu[0] + nb0 + mb0;
          const T Eb = -nb0, Gb = -mb0;
          rhob += Eb * phi<Q, T>(0, T(0), uu) + Gb * (GEN ? phi<Q, T>(0, T(0), usus) : T(lat_w<Q>(0)));
          const T ke = T(-3) * rho * T(lat_w<Q>(0)) * Eb;
          ubx += ke * ux;
          uby += ke * uy;
          ubz += ke * uz;
          if constexpr (GEN) {
            const T kg = T(-3) * rho * T(lat_w<Q>(0)) * Gb;
            usbx += kg * usx;
            usby += kg * usy;
            usbz += kg * usz;
          }
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
          const int j = i + 1;
          const int cx = lat_cx(i), cy = lat_cy(i), cz = lat_cz(i);
          const T cu = cdot(i, ux, uy, uz);
          const T cs = GEN ? cdot(i, usx, usy, usz) : T(0);
          const T Ei = feq_shifted_nz<Q, T>(i, drho, rho, ux, uy, uz, uu);
          const T Ej = feq_shifted_nz<Q, T>(j, drho, rho, ux, uy, uz, uu);
          const T wd = T(lat_w<Q>(i)) * drho;
          const T Gi = GEN ? feq_shifted_nz<Q, T>(i, drho, rho, usx, usy, usz, usus) : wd;
          const T Gj = GEN ? feq_shifted_nz<Q, T>(j, drho, rho, usx, usy, usz, usus) : wd;
          const T ni = f[i] - Ei, nj = f[j] - Ej, mi = f[i] - Gi, mj = f[j] - Gj;
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
          const T sci = GEN ? cdot(i, sbx, sby, sbz) : T(0);  // sbar . c_i; c_j = -c_i
          const T osbi = GEN ? Bw * (mu[i] + sci) : Bw * mu[i], osbj = GEN ? Bw * (mu[j] - sci) : Bw * mu[j];
          const T ofbi = omB * mu[i], ofbj = omB * mu[j];
          if constexpr (GEN) Bbar += mu[i] * (osi - ofi) + mu[j] * (osj - ofj) + sci * (osi - osj);
          else Bbar += mu[i] * (osi - ofi) + mu[j] * (osj - ofj);
          T nbi = TRT ? (-om_a * ofbi - om_b * ofbj) : (-om_a * ofbi);
          T nbj = TRT ? (-om_a * ofbj - om_b * ofbi) : (-om_a * ofbj);
          T mbi, mbj;
          if (p.solid == PSM_SC1) {
            nbi += osbj;
            nbj += osbi;
            mbi = -osbi;
            mbj = -osbj;
          } else if (p.solid == PSM_SC2) {
            mbi = -osbi * inv_tau;
            mbj = -osbj * inv_tau;
          } else {
            mbi = osbj - osbi;
            mbj = osbi - osbj;
          }
          f[i] = mu[i] + nbi + mbi;
          f[j] = mu[j] + nbj + mbj;
          const T Ebi = -nbi, Ebj = -nbj, Gbi = -mbi, Gbj = -mbj;
          if constexpr (GEN)
            rhob += Ebi * phi<Q, T>(i, cu, uu) + Ebj * phi<Q, T>(j, -cu, uu) + Gbi * phi<Q, T>(i, cs, usus) +
                    Gbj * phi<Q, T>(j, -cs, usus);
          else
            rhob += Ebi * phi<Q, T>(i, cu, uu) + Ebj * phi<Q, T>(j, -cu, uu) + (Gbi + Gbj) * T(lat_w<Q>(i));
          // d f^eq_i / d v = rho w_i (3 c_i + 9 (c_i.v) c_i - 3 v), and c_j = -c_i
          const T rw = rho * T(lat_w<Q>(i));
          const T ae = rw * (T(3) * (Ebi - Ebj) + T(9) * cu * (Ebi + Ebj)), be = T(-3) * rw * (Ebi + Ebj);
          ubx += cx ? csign(cx, ae) + be * ux : be * ux;
          uby += cy ? csign(cy, ae) + be * uy : be * uy;
          ubz += cz ? csign(cz, ae) + be * uz : be * uz;
          if constexpr (GEN) {
            const T ag = rw * (T(3) * (Gbi - Gbj) + T(9) * cs * (Gbi + Gbj)), bg = T(-3) * rw * (Gbi + Gbj);
            usbx += cx ? csign(cx, ag) + bg * usx : bg * usx;
            usby += cy ? csign(cy, ag) + bg * usy : bg * usy;
            usbz += cz ? csign(cz, ag) + bg * usz : bg * usz;
          }
        }
        // u = j / rho
        const T jbx = ubx * inv_rho, jby = uby * inv_rho, jbz = ubz * inv_rho;
        rhob -= (ubx * ux + uby * uy + ubz * uz) * inv_rho;
        // ---- lambda^n = fbar + drho/df rhobar + dj/df . jbar ----
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const T l = f[i] + rhob + cdot(i, jbx, jby, jbz);
          static_cast<T*>(p.lout_slot[i])[cell] = l;
          if (GEN && zg.from(lat_cz(i))) {
            // the population is the ghost value g_i(u_in)
            if constexpr (sizeof(T) == 4) {
              au0 += l * p.dghostf[i][0];
              au1 += l * p.dghostf[i][1];
              au2 += l * p.dghostf[i][2];
            } else {
              au0 += l * p.dghost[i][0];
              au1 += l * p.dghost[i][1];
              au2 += l * p.dghost[i][2];
            }
            has_u = true;
          }
        }
        grad[cell] = g_old + (double)(Bbar * Bp);
        if (GEN && owner >= 0) {
          // u_s = omega x r + v  =>  d/d omega = r x usbar
          const T a = usbx, b = usby, c = usbz;
          aw0 = Ry * c - Rz * b;
          aw1 = Rz * a - Rx * c;
          aw2 = Rx * b - Ry * a;
          has_w = true;
        }
      }
      }
    }
    // ---- per-warp partials in T, added into the FP64 block slots in a fixed order ----
    if (!GEN) return;
    if (__any_sync(0xffffffffu, has_w)) {
      for (int bi = 0; bi < nb; ++bi) {
        const bool mine = has_w && owner == bi;
        if (!__any_sync(0xffffffffu, mine)) continue;
        const T v0 = warp_sum(mine ? aw0 : T(0)), v1 = warp_sum(mine ? aw1 : T(0)), v2 = warp_sum(mine ? aw2 : T(0));
        if (lane == 0) {
          s_acc[warp][bi * 3 + 0] += (double)v0;
          s_acc[warp][bi * 3 + 1] += (double)v1;
          s_acc[warp][bi * 3 + 2] += (double)v2;
        }
      }
    }
    if (__any_sync(0xffffffffu, has_u)) {
      const T v0 = warp_sum(au0), v1 = warp_sum(au1), v2 = warp_sum(au2);
      if (lane == 0) {
        s_acc[warp][nb * 3 + 0] += (double)v0;
        s_acc[warp][nb * 3 + 1] += (double)v1;
        s_acc[warp][nb * 3 + 2] += (double)v2;
      }
    }
  };

  TileWalk walk;
  walk.init(p.t, blockIdx.x, gridDim.x);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, walk.advance()) {
    const int x0 = walk.tx * p.t.tx, y0 = walk.ty * p.t.ty, z = walk.z;
    // the forward's classification (fluid-only: B = 0 in the whole tile)
    bool gen = p.delta != nullptr || (p.g.bc_z == PSM_BC_EQ_INLET_OUTLET && (z == 0 || z == p.g.nz - 1));
#pragma unroll
    for (int bi = 0; bi < PSM_MAX_BODIES; ++bi) {
      if (bi < nb) {
        const DevBody& b = p.body[bi];
        gen = gen || (x0 < b.x1 && x0 + p.t.tx > b.x0 && y0 < b.y1 && y0 + p.t.ty > b.y0 && z >= b.z0 && z < b.z1);
      }
    }
    if (gen) {
      if (PART != 1) cell_body(BoolC<true>{}, x0 + lx, y0 + ly, z);
    } else {
      if (PART != 2) cell_body(BoolC<false>{}, x0 + lx, y0 + ly, z);
    }
  }
  if (PART == 1) return;
  __syncthreads();
  __shared__ double blk[NC];
  if ((int)threadIdx.x < ncomp) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += s_acc[w][threadIdx.x];
    blk[threadIdx.x] = s;
  }
  __syncthreads();
  grid_reduce(blk, ncomp, p.partials, p.ticket, p.acc_out);
}

// Initial-state term of dJ/d u_in when f^{n0} = f^eq(rho0, u_in) everywhere:
// sum over cells and populations not taken from a ghost plane of
// lambda^{n0}_i d f^eq_i(rho0, u_in) / d u_in (= d g_i / d u_in).
template <int Q, class T>
__global__ void __launch_bounds__(PSM_THREADS) k_adjoint_init(const __grid_constant__ AdjParams p) {
  const T* lam = static_cast<const T*>(p.lam_in);
  const long long N = p.g.ncell;
  double a[3] = {0, 0, 0};
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(idx / ((long long)p.g.nx * p.g.ny));
    const bool zlo = p.g.bc_z == PSM_BC_EQ_INLET_OUTLET && z == 0;
    const bool zhi = p.g.bc_z == PSM_BC_EQ_INLET_OUTLET && z == p.g.nz - 1;
    for (int i = 0; i < Q; ++i) {
      const int cz = lat_cz(i);
      if ((cz > 0 && zlo) || (cz < 0 && zhi)) continue;
      const double l = (double)lam[(long long)i * N + idx];
      for (int k = 0; k < 3; ++k) a[k] += l * p.dghost[i][k];
    }
  }
  __shared__ double s_w[PSM_THREADS / 32][3];
  __shared__ double blk[3];
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum(a[k]);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < PSM_THREADS / 32; ++w) s += s_w[w][threadIdx.x];
    blk[threadIdx.x] = s;
  }
  __syncthreads();
  grid_reduce(blk, 3, p.partials, p.ticket, p.acc_out);
}

// Split launch of one adjoint step (PSM_ADJ_SPLIT, default on for D3Q19 with
// 4-byte arithmetic; the D3Q27 fluid part would spill at 80 registers): the
// fluid tiles at three blocks per SM, then the general tiles.
#ifndef PSM_ADJ_SPLIT
#define PSM_ADJ_SPLIT 1
#endif
template <class S, int Q, int TRT, int PART>
cudaError_t launch_adjoint_part(const AdjParams& p, cudaStream_t st) {
  static int blocks = persistent_blocks(k_adjoint<S, Q, TRT, PART>, 1ll << 40);
  const int grid = (int)(p.t.ntiles < blocks ? p.t.ntiles : blocks);
  k_adjoint<S, Q, TRT, PART><<<grid, PSM_THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

template <class S, int Q, int TRT>
cudaError_t launch_adjoint_t(const AdjParams& p, cudaStream_t st) {
  if constexpr (PSM_ADJ_SPLIT && sizeof(S) != 8 && Q == 19) {
    const cudaError_t e = launch_adjoint_part<S, Q, TRT, 1>(p, st);
    return e != cudaSuccess ? e : launch_adjoint_part<S, Q, TRT, 2>(p, st);
  } else {
    return launch_adjoint_part<S, Q, TRT, 0>(p, st);
  }
}

template <class S, int Q>
cudaError_t launch_adjoint_q(int trt, const AdjParams& p, cudaStream_t st) {
  return trt ? launch_adjoint_t<S, Q, 1>(p, st) : launch_adjoint_t<S, Q, 0>(p, st);
}

template <class S, int Q>
cudaError_t launch_adjoint_init_q(const AdjParams& p, int blocks, cudaStream_t st) {
  using T = typename Store<S>::T;
  k_adjoint_init<Q, T><<<blocks, PSM_THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace psm

#define PSM_DEFINE_ADJOINT(NAME, S)                                                                      \
  namespace psm {                                                                                        \
  cudaError_t launch_adjoint_##NAME(int Q, int trt, const AdjParams& p, cudaStream_t st) {               \
    return Q == 19 ? launch_adjoint_q<S, 19>(trt, p, st) : launch_adjoint_q<S, 27>(trt, p, st);          \
  }                                                                                                      \
  cudaError_t launch_adjoint_init_##NAME(int Q, const AdjParams& p, int blocks, cudaStream_t st) {       \
    return Q == 19 ? launch_adjoint_init_q<S, 19>(p, blocks, st) : launch_adjoint_init_q<S, 27>(p, blocks, st); \
  }                                                                                                      \
  }
