// Host voxelisers of analytic bodies into the brick-packed super-sampled
// geometry field of Sec. 3 (layout documented at psm_geom_field in psm.h).
// The paper voxelises a triangle mesh once on the CPU and copies the binary
// field to the GPU once; here analytic inside tests stand in for the mesh.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/psm.h"

namespace psm {
int set_error(int code, const char* msg);
}

namespace {

enum Kind { SPHERE = 0, ELLIPSOID = 1, BOX = 2, ROTOR = 3 };

struct Shape {
  Kind kind;
  double p[3];
  psm_rotor rotor;
};

bool inside(const Shape& S, double x, double y, double z) {
  switch (S.kind) {
    case SPHERE: return x * x + y * y + z * z <= S.p[0] * S.p[0];
    case ELLIPSOID: {
      const double a = x / S.p[0], b = y / S.p[1], c = z / S.p[2];
      return a * a + b * b + c * c <= 1.0;
    }
    case BOX: return std::fabs(x) <= S.p[0] && std::fabs(y) <= S.p[1] && std::fabs(z) <= S.p[2];
    default: break;
  }
  const psm_rotor& R = S.rotor;
  const double PI = 3.14159265358979323846;
  const double r = std::sqrt(x * x + y * y);
  if (r <= R.r_hub && std::fabs(z) <= 0.5 * R.hub_len) return true;
  if (r < R.r_hub || r > R.r_hub + R.span) return false;
  const double phi = std::atan2(y, x);
  const double beta = (R.pitch_root_deg - R.twist_deg * (r - R.r_hub) / R.span) * (PI / 180.0) * double(R.hand);
  const double cb = std::cos(beta), sb = std::sin(beta);
  const double ha = 0.5 * R.chord, hb = 0.5 * R.thickness;
  for (int k = 0; k < R.n_blades; ++k) {
    double dphi = phi - (R.phase + 2.0 * PI * double(k) / double(R.n_blades));
    dphi = dphi - 2.0 * PI * std::floor((dphi + PI) / (2.0 * PI));
    const double t = r * dphi;
    const double xi = t * cb + z * sb;
    const double eta = -t * sb + z * cb;
    const double qa = xi / ha, qb = eta / hb;
    if (qa * qa + qb * qb <= 1.0) return true;
  }
  return false;
}

void half_extent(const Shape& S, double he[3]) {
  if (S.kind == SPHERE) {
    he[0] = he[1] = he[2] = S.p[0];
  } else if (S.kind == ELLIPSOID || S.kind == BOX) {
    for (int k = 0; k < 3; ++k) he[k] = S.p[k];
  } else {
    const psm_rotor& R = S.rotor;
    he[0] = he[1] = R.r_hub + R.span;
    he[2] = std::max(0.5 * R.hub_len, 0.5 * std::sqrt(R.chord * R.chord + R.thickness * R.thickness));
  }
}

int voxelize(const Shape& S, int s, psm_geom_field* out) {
  if (!out) return psm::set_error(PSM_ERR_ARG, "voxelize: NULL output");
  out->bricks = nullptr;
  if (s < 0 || s > 3) return psm::set_error(PSM_ERR_ARG, "super-sampling depth s must be 0..3");
  double he[3];
  half_extent(S, he);
  int64_t dims[3];
  double lo[3];
  for (int k = 0; k < 3; ++k) {
    if (!(he[k] > 0.0) || !std::isfinite(he[k]) || he[k] > 1e5)
      return psm::set_error(PSM_ERR_ARG, "body extent must be finite, > 0 and < 1e5 cells");
    const int64_t m = (int64_t)std::floor(he[k]) + 2;
    dims[k] = 2 * m;
    lo[k] = -(double)m;
  }
  const int n = 1 << s;
  const int wpb = s == 3 ? 8 : 1;
  const size_t nbricks = (size_t)dims[0] * dims[1] * dims[2];
  uint64_t* bricks = static_cast<uint64_t*>(std::calloc(nbricks * wpb, sizeof(uint64_t)));
  if (!bricks) return psm::set_error(PSM_ERR_OOM, "geometry field allocation failed");
  const double h = 1.0 / double(n);
  auto work = [&](int64_t gz0, int64_t gz1) {
    for (int64_t gz = gz0; gz < gz1; ++gz)
      for (int64_t gy = 0; gy < dims[1]; ++gy)
        for (int64_t gx = 0; gx < dims[0]; ++gx) {
          uint64_t* br = bricks + ((size_t)(gz * dims[1] + gy) * dims[0] + gx) * wpb;
          for (int sz = 0; sz < n; ++sz)
            for (int sy = 0; sy < n; ++sy)
              for (int sx = 0; sx < n; ++sx) {
                const int64_t ax = gx * n + sx, ay = gy * n + sy, az = gz * n + sz;
                const double x = lo[0] + (double(ax) + 0.5) * h;
                const double y = lo[1] + (double(ay) + 0.5) * h;
                const double z = lo[2] + (double(az) + 0.5) * h;
                if (inside(S, x, y, z)) {
                  const int bit = (sz * n + sy) * n + sx;
                  br[bit >> 6] |= 1ull << (bit & 63);
                }
              }
        }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if ((int64_t)nt > dims[2]) nt = (unsigned)dims[2];
  std::vector<std::thread> th;
  try {
    for (unsigned t = 0; t < nt; ++t) {
      const int64_t a = dims[2] * t / nt, b = dims[2] * (t + 1) / nt;
      th.emplace_back(work, a, b);
    }
  } catch (...) {
    for (auto& x : th) x.join();
    std::free(bricks);
    return psm::set_error(PSM_ERR_OOM, "could not start voxeliser threads");
  }
  for (auto& x : th) x.join();
  out->bricks = bricks;
  out->gx = dims[0];
  out->gy = dims[1];
  out->gz = dims[2];
  out->s = s;
  for (int k = 0; k < 3; ++k) out->lo[k] = lo[k];
  return PSM_OK;
}

}  // namespace

extern "C" {

int psm_geom_voxelize_sphere(double r, int s, psm_geom_field* out) {
  if (!(r > 0.0)) return psm::set_error(PSM_ERR_ARG, "sphere radius must be > 0");
  Shape S{};
  S.kind = SPHERE;
  S.p[0] = r;
  return voxelize(S, s, out);
}

int psm_geom_voxelize_ellipsoid(double a, double b, double c, int s, psm_geom_field* out) {
  if (!(a > 0.0 && b > 0.0 && c > 0.0)) return psm::set_error(PSM_ERR_ARG, "semi-axes must be > 0");
  Shape S{};
  S.kind = ELLIPSOID;
  S.p[0] = a;
  S.p[1] = b;
  S.p[2] = c;
  return voxelize(S, s, out);
}

int psm_geom_voxelize_box(double hx, double hy, double hz, int s, psm_geom_field* out) {
  if (!(hx > 0.0 && hy > 0.0 && hz > 0.0)) return psm::set_error(PSM_ERR_ARG, "half extents must be > 0");
  Shape S{};
  S.kind = BOX;
  S.p[0] = hx;
  S.p[1] = hy;
  S.p[2] = hz;
  return voxelize(S, s, out);
}

int psm_geom_voxelize_rotor(const psm_rotor* rotor, int s, psm_geom_field* out) {
  if (!rotor) return psm::set_error(PSM_ERR_ARG, "rotor: NULL argument");
  const psm_rotor& R = *rotor;
  if (!(R.r_hub > 0 && R.hub_len > 0 && R.span > 0 && R.chord > 0 && R.thickness > 0) || R.n_blades < 0 ||
      R.n_blades > 64 || (R.hand != 1 && R.hand != -1))
    return psm::set_error(PSM_ERR_ARG, "rotor: sizes must be > 0, 0 <= n_blades <= 64, hand = +-1");
  Shape S{};
  S.kind = ROTOR;
  S.rotor = R;
  return voxelize(S, s, out);
}

int psm_geom_free(psm_geom_field* field) {
  if (!field) return psm::set_error(PSM_ERR_ARG, "psm_geom_free: NULL argument");
  std::free(const_cast<uint64_t*>(field->bricks));
  field->bricks = nullptr;
  return PSM_OK;
}

}  // extern "C"
