// Voxelisation of a closed triangle mesh into the super-sampled binary
// geometry field of Sec. 3 (the paper voxelises the body's surface mesh once
// and keeps the binary field), on the GPU.
//
// A sub-cell is inside iff a ray from its centre in the +x direction crosses
// the surface an odd number of times, decided in exact integer arithmetic:
//   * field box [lo, lo + dims): lo = floor(min v) - 1, lo + dims = ceil(max v) + 1
//     per axis (whole cells), dims <= 2^(19 - s);
//   * vertex coordinates relative to lo quantised to integers in units of
//     2^-(s+8) cells, rounded half away from zero; the centre of sub-cell a is
//     at 256 a + 128;
//   * the ray hits a triangle's (y, z) projection when the three edge
//     orientations share one strict sign, where a zero orientation takes the
//     sign it would have with the centre moved by (delta^2, delta) in (y, z),
//     delta -> 0+ (a point on a shared edge or vertex falls on one side only);
//   * a hit counts when the crossing lies at or ahead of the centre in x.
// Work: one thread per sub-cell row (y, z); triangles are binned by the rows
// their projection's bounding box covers (tiles of 16 x 16 rows); each row
// finds, per hit triangle, how many of its centres see the crossing (binary
// search on an exact, monotone integer test) and XORs that prefix into the
// row; rows are OR-ed into the bricks.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "psm_internal.h"

namespace psm {
int set_error(int code, const char* msg);
}

namespace {

constexpr int TILE = 16;      // rows per tile side
constexpr int MAX_HITS = 256; // crossings one row may collect

struct TriQ {
  long long v[3][3];  // quantised vertices
  int y0, y1, z0, z1; // rows (sub-cell indices) the projection's bounding box covers, inclusive
};

__device__ __forceinline__ long long qcoord(float c, double lo, double scale) {
  return llround(((double)c - lo) * scale);
}

// rows a whose centre 256 a + 128 lies in [mn, mx], clamped to [0, n)
__device__ __forceinline__ void row_range(long long mn, long long mx, int n, int& a0, int& a1) {
  long long lo = (mn - 128 + 255) >> 8;  // ceil((mn - 128) / 256)
  long long hi = (mx - 128) >> 8;        // floor((mx - 128) / 256)
  if (lo < 0) lo = 0;
  if (hi > n - 1) hi = n - 1;
  a0 = (int)lo;
  a1 = (int)hi;
}

__global__ void k_mesh_prepare(const float* __restrict__ vert, const int* __restrict__ tri, long long nt, double lo0,
                               double lo1, double lo2, double scale, int ny, int nz, TriQ* __restrict__ out,
                               unsigned* __restrict__ cnt, int tiles_y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
    TriQ q;
    const double lo[3] = {lo0, lo1, lo2};
    for (int c = 0; c < 3; ++c) {
      const int vi = tri[3 * t + c];
      for (int k = 0; k < 3; ++k) q.v[c][k] = qcoord(vert[3 * (long long)vi + k], lo[k], scale);
    }
    const long long ymn = min(q.v[0][1], min(q.v[1][1], q.v[2][1])), ymx = max(q.v[0][1], max(q.v[1][1], q.v[2][1]));
    const long long zmn = min(q.v[0][2], min(q.v[1][2], q.v[2][2])), zmx = max(q.v[0][2], max(q.v[1][2], q.v[2][2]));
    row_range(ymn, ymx, ny, q.y0, q.y1);
    row_range(zmn, zmx, nz, q.z0, q.z1);
    out[t] = q;
    if (q.y0 > q.y1 || q.z0 > q.z1) continue;
    for (int tz = q.z0 / TILE; tz <= q.z1 / TILE; ++tz)
      for (int ty = q.y0 / TILE; ty <= q.y1 / TILE; ++ty) atomicAdd(&cnt[tz * tiles_y + ty], 1u);
  }
}

__global__ void k_mesh_bin(const TriQ* __restrict__ tq, long long nt, unsigned* __restrict__ cursor,
                           unsigned* __restrict__ list, int tiles_y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
    const TriQ& q = tq[t];
    if (q.y0 > q.y1 || q.z0 > q.z1) continue;
    for (int tz = q.z0 / TILE; tz <= q.z1 / TILE; ++tz)
      for (int ty = q.y0 / TILE; ty <= q.y1 / TILE; ++ty) {
        const unsigned pos = atomicAdd(&cursor[tz * tiles_y + ty], 1u);
        list[pos] = (unsigned)t;
      }
  }
}

// sign of the (y, z) orientation of the centre against the directed edge
// a -> b, with the centre moved by (delta^2, delta)
__device__ __forceinline__ int edge_sign(const long long* a, const long long* b, long long py, long long pz) {
  const long long ey = b[1] - a[1], ez = b[2] - a[2];
  const long long o = ey * (pz - a[2]) - ez * (py - a[1]);
  if (o != 0) return o > 0 ? 1 : -1;
  if (ey != 0) return ey > 0 ? 1 : -1;
  if (ez != 0) return ez < 0 ? 1 : -1;
  return 0;
}

__global__ void k_mesh_rows(const TriQ* __restrict__ tq, const unsigned* __restrict__ start,
                            const unsigned* __restrict__ list, int nxs, int ny, int nz, int tiles_y, int s,
                            unsigned long long* __restrict__ bricks, int gx, int gy, int wpb, int* __restrict__ err) {
  const long long nrows = (long long)ny * nz;
  const int n = 1 << s;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrows; r += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const long long py = 256ll * j + 128, pz = 256ll * k + 128;
    const int tile = (k / TILE) * tiles_y + j / TILE;
    int m[MAX_HITS];
    int nh = 0;
    for (unsigned e = start[tile]; e < start[tile + 1]; ++e) {
      const TriQ& q = tq[list[e]];
      if (j < q.y0 || j > q.y1 || k < q.z0 || k > q.z1) continue;
      const long long *A = q.v[0], *B = q.v[1], *C = q.v[2];
      const int s1 = edge_sign(A, B, py, pz), s2 = edge_sign(B, C, py, pz), s3 = edge_sign(C, A, py, pz);
      if (s1 == 0 || s1 != s2 || s2 != s3) continue;
      const long long e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      const long long e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      const long long nx = e1[1] * e2[2] - e1[2] * e2[1];
      const long long nyv = e1[2] * e2[0] - e1[0] * e2[2];
      const long long nzv = e1[0] * e2[1] - e1[1] * e2[0];
      // the crossing is at or ahead of centre i (x = 256 i + 128) iff
      // sgn(nx) (D0 - 256 nx i) >= 0 with D0 = n . (A - (128, py, pz)):
      // a - b i >= 0, decreasing in i; m = the number of such i in [0, nxs)
      const __int128 D0 = (__int128)nx * (A[0] - 128) + (__int128)nyv * (A[1] - py) + (__int128)nzv * (A[2] - pz);
      const __int128 a = nx > 0 ? D0 : -D0;
      const __int128 b = (__int128)(nx > 0 ? nx : -nx) * 256;
      int lo = -1, hi = nxs;  // invariant: a - b lo >= 0 (or lo = -1), a - b hi < 0 (or hi = nxs)
      while (hi - lo > 1) {
        const int mid = (int)(((long long)lo + hi) >> 1);
        if (a - b * mid >= 0) lo = mid;
        else hi = mid;
      }
      if (nh == MAX_HITS) {
        atomicExch(err, 1);
        break;
      }
      m[nh++] = lo + 1;
    }
    if (nh == 0) continue;
    // row bits, word by word: bit i is the parity of #{hits with i < m}
    const int nw = (nxs + 63) >> 6;
    const int sy = j & (n - 1), sz = k & (n - 1), cy = j >> s, cz = k >> s;
    for (int w = 0; w < nw; ++w) {
      unsigned long long word = 0ull;
      for (int h = 0; h < nh; ++h) {
        const int c = m[h] - 64 * w;
        if (c <= 0) continue;
        word ^= c >= 64 ? ~0ull : ((1ull << c) - 1ull);
      }
      if (!word) continue;
      // coarse cells covered by this word: n bits each
      for (int cx = (64 * w) >> s; cx <= (64 * w + 63) >> s && cx < gx; ++cx) {
        const int b0 = cx * n - 64 * w;  // first bit of the cell in the word (b0 >= 0, n <= 8)
        const unsigned long long bits = (word >> b0) & ((1ull << n) - 1ull);
        if (!bits) continue;
        unsigned long long* brick = bricks + (((long long)cz * gy + cy) * gx + cx) * wpb;
        const int bit = (sz * n + sy) * n;  // (sz n + sy) n + sx with sx = 0 .. n - 1
        atomicOr(brick + (bit >> 6), bits << (bit & 63));
      }
    }
  }
}

int mesh_fail(int code, const char* msg) { return psm::set_error(code, msg); }

}  // namespace

extern "C" int psm_geom_voxelize_mesh(const float* vertices, int64_t nv, const int32_t* triangles, int64_t nt, int s,
                                      psm_geom_field* out) {
  if (!out) return mesh_fail(PSM_ERR_ARG, "psm_geom_voxelize_mesh: NULL output");
  out->bricks = nullptr;
  if (!vertices || !triangles) return mesh_fail(PSM_ERR_ARG, "psm_geom_voxelize_mesh: NULL argument");
  if (s < 0 || s > 3) return mesh_fail(PSM_ERR_ARG, "super-sampling depth s must be 0..3");
  if (nv < 3 || nt < 1 || nv > (1ll << 31) - 1 || nt > (1ll << 31) - 1)
    return mesh_fail(PSM_ERR_ARG, "mesh needs 3 <= vertices < 2^31 and 1 <= triangles < 2^31");
  // host copies (the inputs may live on the device; host inputs need no GPU
  // for the argument checks)
  auto fetch = [](void* dst, const void* src, size_t bytes) -> bool {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess &&
        (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged))
      return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaGetLastError();  // a host pointer (or no device): not an error
    std::memcpy(dst, src, bytes);
    return true;
  };
  std::vector<float> hv((size_t)nv * 3);
  std::vector<int32_t> ht((size_t)nt * 3);
  if (!fetch(hv.data(), vertices, sizeof(float) * hv.size()) || !fetch(ht.data(), triangles, sizeof(int32_t) * ht.size()))
    return mesh_fail(PSM_ERR_CUDA, "mesh read failed");
  for (int32_t i : ht)
    if (i < 0 || i >= nv) return mesh_fail(PSM_ERR_ARG, "triangle vertex index out of range");
  // closed: every undirected edge is shared by an even number of triangles
  {
    std::vector<uint64_t> edges;
    edges.reserve((size_t)nt * 3);
    for (int64_t t = 0; t < nt; ++t)
      for (int c = 0; c < 3; ++c) {
        const uint32_t a = (uint32_t)ht[3 * t + c], b = (uint32_t)ht[3 * t + (c + 1) % 3];
        if (a == b) return mesh_fail(PSM_ERR_ARG, "degenerate triangle (repeated vertex index)");
        edges.push_back(((uint64_t)std::min(a, b) << 32) | std::max(a, b));
      }
    std::sort(edges.begin(), edges.end());
    for (size_t i = 0; i < edges.size();) {
      size_t k = i;
      while (k < edges.size() && edges[k] == edges[i]) ++k;
      if ((k - i) & 1) return mesh_fail(PSM_ERR_ARG, "mesh is not closed (an edge has an odd number of triangles)");
      i = k;
    }
  }
  int64_t dims[3];
  double lo[3];
  for (int k = 0; k < 3; ++k) {
    double mn = 1e300, mx = -1e300;
    for (int64_t i = 0; i < nv; ++i) {
      const double c = (double)hv[3 * i + k];
      if (!std::isfinite(c)) return mesh_fail(PSM_ERR_ARG, "non-finite vertex coordinate");
      mn = std::min(mn, c);
      mx = std::max(mx, c);
    }
    lo[k] = std::floor(mn) - 1.0;
    dims[k] = (int64_t)(std::ceil(mx) + 1.0 - lo[k]);
    if (dims[k] > ((int64_t)1 << (19 - s))) return mesh_fail(PSM_ERR_ARG, "mesh extent exceeds 2^(19-s) cells");
  }
  const int n = 1 << s;
  const int wpb = s == 3 ? 8 : 1;
  const int nxs = (int)(dims[0] * n), ny = (int)(dims[1] * n), nz = (int)(dims[2] * n);
  const int tiles_y = (ny + TILE - 1) / TILE, tiles_z = (nz + TILE - 1) / TILE;
  const size_t ntiles = (size_t)tiles_y * tiles_z;
  const size_t nwords = (size_t)dims[0] * dims[1] * dims[2] * wpb;

  float* dv = nullptr;
  int* dt = nullptr;
  TriQ* dq = nullptr;
  unsigned *dcnt = nullptr, *dlist = nullptr;
  unsigned long long* dbr = nullptr;
  int* derr = nullptr;
  auto release = [&]() {
    cudaFree(dv);
    cudaFree(dt);
    cudaFree(dq);
    cudaFree(dcnt);
    cudaFree(dlist);
    cudaFree(dbr);
    cudaFree(derr);
  };
  cudaError_t e = cudaMalloc(&dv, sizeof(float) * hv.size());
  if (e == cudaSuccess) e = cudaMalloc(&dt, sizeof(int) * ht.size());
  if (e == cudaSuccess) e = cudaMalloc(&dq, sizeof(TriQ) * (size_t)nt);
  if (e == cudaSuccess) e = cudaMalloc(&dcnt, sizeof(unsigned) * (ntiles + 1));
  if (e == cudaSuccess) e = cudaMalloc(&dbr, sizeof(unsigned long long) * nwords);
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dv, hv.data(), sizeof(float) * hv.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt, ht.data(), sizeof(int) * ht.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dcnt, 0, sizeof(unsigned) * (ntiles + 1));
  if (e == cudaSuccess) e = cudaMemset(dbr, 0, sizeof(unsigned long long) * nwords);
  if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
  if (e != cudaSuccess) {
    release();
    return mesh_fail(e == cudaErrorMemoryAllocation ? PSM_ERR_OOM : PSM_ERR_CUDA, "mesh voxeliser setup failed");
  }
  const double scale = std::ldexp(1.0, s + 8);
  const int tb = 256;
  const int tgrid = (int)std::min<int64_t>((nt + tb - 1) / tb, 4096);
  k_mesh_prepare<<<tgrid, tb>>>(dv, dt, nt, lo[0], lo[1], lo[2], scale, ny, nz, dq, dcnt, tiles_y);
  // bin offsets: exclusive scan of the tile counts on the host
  std::vector<unsigned> cnt(ntiles + 1, 0u);
  e = cudaMemcpy(cnt.data(), dcnt, sizeof(unsigned) * ntiles, cudaMemcpyDeviceToHost);
  uint64_t total = 0;
  for (size_t t = 0; t < ntiles; ++t) {
    const unsigned c = cnt[t];
    cnt[t] = (unsigned)total;
    total += c;
  }
  cnt[ntiles] = (unsigned)total;
  if (e == cudaSuccess && total > 0xffffffffull) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = cudaMalloc(&dlist, sizeof(unsigned) * (size_t)std::max<uint64_t>(total, 1));
  unsigned* dstart = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&dstart, sizeof(unsigned) * (ntiles + 1));
  if (e == cudaSuccess) e = cudaMemcpy(dstart, cnt.data(), sizeof(unsigned) * (ntiles + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dcnt, cnt.data(), sizeof(unsigned) * ntiles, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_mesh_bin<<<tgrid, tb>>>(dq, nt, dcnt, dlist, tiles_y);
    const long long nrows = (long long)ny * nz;
    const int rgrid = (int)std::min<long long>((nrows + tb - 1) / tb, 65536);
    k_mesh_rows<<<rgrid, tb>>>(dq, dstart, dlist, nxs, ny, nz, tiles_y, s, dbr, (int)dims[0], (int)dims[1], wpb,
                               derr);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  uint64_t* bricks = nullptr;
  if (e == cudaSuccess && !herr) {
    bricks = static_cast<uint64_t*>(std::calloc(nwords, sizeof(uint64_t)));
    if (!bricks) {
      cudaFree(dstart);
      release();
      return mesh_fail(PSM_ERR_OOM, "geometry field allocation failed");
    }
    e = cudaMemcpy(bricks, dbr, sizeof(uint64_t) * nwords, cudaMemcpyDeviceToHost);
  }
  cudaFree(dstart);
  release();
  if (e != cudaSuccess) {
    std::free(bricks);
    return mesh_fail(PSM_ERR_CUDA, "mesh voxeliser kernels failed");
  }
  if (herr) return mesh_fail(PSM_ERR_UNSUPPORTED, "more than 256 surface crossings along one sub-cell row");
  out->bricks = bricks;
  out->gx = dims[0];
  out->gy = dims[1];
  out->gz = dims[2];
  out->s = s;
  for (int k = 0; k < 3; ++k) out->lo[k] = lo[k];
  return PSM_OK;
}
