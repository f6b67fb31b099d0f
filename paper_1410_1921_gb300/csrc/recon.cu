// recon.cu -- random pore-sphere reconstruction (Sec. 2).
//
// Host: the sequential acceptance loop.  Candidate spheres come from one
// SplitMix64 stream (Steele, Lea & Flood 2014) in a fixed draw order: for
// every sphere after the first an "overlap required" flag (u < p0), then per
// trial the centre x, y, z (uniform over the box, voxel units) and the
// diameter.  A trial is accepted when, against every placed sphere, the
// overlapped volume is at most xi times each sphere's own volume, and, if
// overlap is required, it overlaps at least one of them (steps 1-2).  The
// test visits only spheres in neighbouring cells of a uniform grid whose cell
// edge is the largest possible diameter, so it costs O(1) per trial.
//
// Device: accepted spheres are rasterised in batches.  Every voxel records
// the smallest index of the spheres covering it (atomicMin); the number of
// voxels a sphere k covers first is then the count of voxels owned by k, and
// the porosity after each acceptance is a prefix sum of those counts.  The
// reconstruction stops at the first acceptance that reaches the target
// porosity (step 3) and the mask is "owner <= that sphere".
//
// The decisions are floating-point comparisons, so their arithmetic is
// fixed: every distance, volume and voxel test below is a sequence of
// individually rounded IEEE double operations (no fused multiply-add: host
// code is compiled with -ffp-contract=off, device code uses the _rn
// intrinsics) and libm's log, cos and sqrt for the normal draws.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace om {
namespace {

constexpr double kPi = 3.14159265358979323846;

struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
};

struct Ball {
  double c[3];
  double r;
};

double ball_volume(double r) { return (4.0 * kPi / 3.0) * (r * r * r); }

// volume shared by balls of radii r1, r2 whose centres are `dist` apart
double overlap_volume(double r1, double r2, double dist) {
  const double rs = r1 + r2;
  if (dist >= rs) return 0.0;
  if (dist <= std::fabs(r1 - r2)) return ball_volume(std::min(r1, r2));
  const double h = rs - dist;
  const double dr = r1 - r2;
  const double q = dist * dist + 2.0 * dist * rs - 3.0 * (dr * dr);
  return kPi * (h * h) * q / (12.0 * dist);
}

double periodic_gap(double d, int n) {
  if (d > 0.5 * n) return d - n;
  if (d < -0.5 * n) return d + n;
  return d;
}

struct Placer {
  om_domain dom;
  om_recon_params p;
  SplitMix64 rng;
  std::vector<Ball> balls;
  // uniform grid of cells, each at least one maximal diameter wide
  int gx = 1, gy = 1, gz = 1;
  double hx = 1, hy = 1, hz = 1;
  std::vector<std::vector<int32_t>> cells;
  int64_t trials = 0;

  void init(uint64_t seed) {
    rng.s = seed;
    const double dmax = (p.dist == 1 ? p.mean_d_nm + p.sd_d_nm : p.dmax_nm) / dom.dx_nm;
    const double h = std::max(1.0, dmax);
    gx = std::max(1, (int)(dom.nx / h));
    gy = std::max(1, (int)(dom.ny / h));
    gz = std::max(1, (int)(dom.nz / h));
    hx = (double)dom.nx / gx;
    hy = (double)dom.ny / gy;
    hz = (double)dom.nz / gz;
    cells.assign((size_t)gx * gy * gz, {});
  }
  int cell_of(double v, double h, int g) const { return std::min(g - 1, std::max(0, (int)(v / h))); }

  double draw_diameter() {
    if (p.dist == 1) {
      const double u = rng.uniform();
      return (p.mean_d_nm - p.sd_d_nm) + (2.0 * p.sd_d_nm) * u;
    }
    const double u1 = rng.uniform();
    const double u2 = rng.uniform();
    const double z = std::sqrt(-2.0 * std::log(1.0 - u1)) * std::cos(2.0 * kPi * u2);
    double d = p.mean_d_nm + p.sd_d_nm * z;
    if (d < p.dmin_nm) d = p.dmin_nm;
    if (d > p.dmax_nm) d = p.dmax_nm;
    return d;
  }

  // tolerance and overlap-requirement test of a trial against placed balls
  bool acceptable(const Ball& t, bool must_touch) const {
    const double vt = ball_volume(t.r);
    bool touched = false;
    const int ix = cell_of(t.c[0], hx, gx), iy = cell_of(t.c[1], hy, gy), iz = cell_of(t.c[2], hz, gz);
    int ys[3], zs[3], ny = 0, nz = 0;
    for (int d = -1; d <= 1; ++d) {
      int y = ((iy + d) % gy + gy) % gy, z = ((iz + d) % gz + gz) % gz;
      if (std::find(ys, ys + ny, y) == ys + ny) ys[ny++] = y;
      if (std::find(zs, zs + nz, z) == zs + nz) zs[nz++] = z;
    }
    for (int x = std::max(0, ix - 1); x <= std::min(gx - 1, ix + 1); ++x)
      for (int a = 0; a < ny; ++a)
        for (int b = 0; b < nz; ++b)
          for (int32_t k : cells[((size_t)x * gy + ys[a]) * gz + zs[b]]) {
            const Ball& s = balls[k];
            const double dx = t.c[0] - s.c[0];
            const double dy = periodic_gap(t.c[1] - s.c[1], dom.ny);
            const double dz = periodic_gap(t.c[2] - s.c[2], dom.nz);
            const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
            const double v = overlap_volume(t.r, s.r, dist);
            if (v > 0.0) touched = true;
            if (v / vt > p.overlap_tol || v / ball_volume(s.r) > p.overlap_tol) return false;
          }
    return touched || !must_touch;
  }

  void add(const Ball& b) {
    const int ix = cell_of(b.c[0], hx, gx), iy = cell_of(b.c[1], hy, gy), iz = cell_of(b.c[2], hz, gz);
    cells[((size_t)ix * gy + iy) * gz + iz].push_back((int32_t)balls.size());
    balls.push_back(b);
  }

  // place the next sphere (steps 1-2); false when the trial cap is hit
  bool place_next() {
    const bool first = balls.empty();
    const bool must_touch = first ? false : rng.uniform() < p.p_overlap;
    for (;;) {
      if (trials >= p.max_trials) return false;
      ++trials;
      Ball t;
      t.c[0] = rng.uniform() * dom.nx;
      t.c[1] = rng.uniform() * dom.ny;
      t.c[2] = rng.uniform() * dom.nz;
      t.r = 0.5 * (draw_diameter() / dom.dx_nm);
      if (first || acceptable(t, must_touch)) {
        add(t);
        return true;
      }
    }
  }
};

// ------------------------------------------------------------------ device
struct DevBall {
  double cx, cy, cz, r;
  int x0, x1, y0, y1, z0, z1;  // bounding box (y, z may wrap)
};

__device__ __forceinline__ bool voxel_in_ball(int vx, int vy, int vz, const DevBall& b, int ny, int nz) {
  const double ddx = __dsub_rn(__dadd_rn((double)vx, 0.5), b.cx);
  const double r2 = __dmul_rn(b.r, b.r);
  const double xx = __dmul_rn(ddx, ddx);
  for (int ky = -1; ky <= 1; ++ky) {
    const double ddy = __dsub_rn(__dadd_rn((double)vy, 0.5), __dadd_rn(b.cy, (double)(ky * ny)));
    const double xy = __dadd_rn(xx, __dmul_rn(ddy, ddy));
    for (int kz = -1; kz <= 1; ++kz) {
      const double ddz = __dsub_rn(__dadd_rn((double)vz, 0.5), __dadd_rn(b.cz, (double)(kz * nz)));
      if (__dadd_rn(xy, __dmul_rn(ddz, ddz)) <= r2) return true;
    }
  }
  return false;
}

__global__ void raster_balls(const DevBall* balls, int k0, int nx, int ny, int nz, int* owner) {
  const DevBall b = balls[blockIdx.x];
  const int k = k0 + (int)blockIdx.x;
  const int bx = b.x1 - b.x0 + 1, by = b.y1 - b.y0 + 1, bz = b.z1 - b.z0 + 1;
  const int64_t total = (int64_t)bx * by * bz;
  for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
    const int zz = (int)(i % bz), yy = (int)((i / bz) % by), xx = (int)(i / ((int64_t)bz * by));
    const int x = b.x0 + xx;
    int y = (b.y0 + yy) % ny;
    if (y < 0) y += ny;
    int z = (b.z0 + zz) % nz;
    if (z < 0) z += nz;
    if (voxel_in_ball(x, y, z, b, ny, nz)) atomicMin(owner + ((int64_t)x * ny + y) * nz + z, k);
  }
}

__global__ void count_first_cover(const int* owner, int64_t N, int k0, int k1, unsigned long long* cnt) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int o = owner[v];
    if (o >= k0 && o < k1) atomicAdd(cnt + (o - k0), 1ull);
  }
}

__global__ void owner_to_mask(const int* owner, int64_t N, int kstop, uint8_t* mask) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    mask[v] = owner[v] <= kstop ? 1 : 0;
}

__global__ void fill_int(int* p, int64_t n, int val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = val;
}

DevBall to_dev(const Ball& b, const om_domain& d) {
  DevBall o;
  o.cx = b.c[0];
  o.cy = b.c[1];
  o.cz = b.c[2];
  o.r = b.r;
  o.x0 = std::max(0, (int)std::floor(b.c[0] - b.r) - 1);
  o.x1 = std::min(d.nx - 1, (int)std::ceil(b.c[0] + b.r) + 1);
  o.y0 = (int)std::floor(b.c[1] - b.r) - 1;
  o.y1 = (int)std::ceil(b.c[1] + b.r) + 1;
  if (o.y1 - o.y0 + 1 > d.ny) { o.y0 = 0; o.y1 = d.ny - 1; }
  o.z0 = (int)std::floor(b.c[2] - b.r) - 1;
  o.z1 = (int)std::ceil(b.c[2] + b.r) + 1;
  if (o.z1 - o.z0 + 1 > d.nz) { o.z0 = 0; o.z1 = d.nz - 1; }
  if (o.x1 < o.x0) o.x1 = o.x0 - 1;  // empty in x (cannot happen for centres in the box)
  return o;
}

om_status reconstruct_impl(uint64_t seed, const om_domain& d, const om_recon_params& p, uint8_t* mask_dev,
                           double* eps_out, int64_t* nsph_out, cudaStream_t s) {
  OM_TRY(check_domain(d));
  if (!(p.porosity > 0.0 && p.porosity <= 1.0)) return fail(OM_EINVAL, "porosity must be in (0, 1]");
  if (!(p.overlap_tol >= 0.0) || !(p.p_overlap >= 0.0 && p.p_overlap <= 1.0) || p.max_trials <= 0)
    return fail(OM_EINVAL, "bad overlap tolerance, p_overlap or max_trials");
  if (p.dist != 0 && p.dist != 1) return fail(OM_EINVAL, "dist must be 0 (normal) or 1 (uniform)");
  if (p.dist == 0 && !(p.dmin_nm > 0.0 && p.dmax_nm >= p.dmin_nm))
    return fail(OM_EINVAL, "need 0 < dmin_nm <= dmax_nm");
  if (p.dist == 1 && !(p.mean_d_nm - p.sd_d_nm > 0.0)) return fail(OM_EINVAL, "uniform diameters must be positive");
  const int64_t N = voxels(d);
  Placer pl;
  pl.dom = d;
  pl.p = p;
  pl.init(seed);

  DevBuf<int> owner;
  OM_TRY(owner.alloc(N));
  fill_int<<<1216, 256, 0, s>>>(owner.p, N, 0x7fffffff);
  OM_CUDA(cudaGetLastError());

  const double rmean = 0.5 * p.mean_d_nm / d.dx_nm;
  const double vmean = std::max(1.0, ball_volume(rmean));
  int64_t covered = 0;
  int kstop = -1;
  bool infeasible = false;
  std::vector<DevBall> host_balls;
  std::vector<unsigned long long> cnt;
  DevBuf<DevBall> dballs;
  DevBuf<unsigned long long> dcnt;
  while (kstop < 0 && !infeasible) {
    const double need = p.porosity * (double)N - (double)covered;
    int64_t chunk = (int64_t)std::ceil(1.5 * std::max(0.0, need) / vmean) + 16;
    chunk = std::min<int64_t>(chunk, 1 << 18);
    const int k0 = (int)pl.balls.size();
    for (int64_t i = 0; i < chunk; ++i)
      if (!pl.place_next()) {
        infeasible = true;
        break;
      }
    const int k1 = (int)pl.balls.size();
    if (k1 == k0) break;
    host_balls.resize(k1 - k0);
    for (int k = k0; k < k1; ++k) host_balls[k - k0] = to_dev(pl.balls[k], d);
    OM_TRY(dballs.alloc(k1 - k0));
    OM_TRY(dcnt.alloc(k1 - k0));
    OM_CUDA(cudaMemcpyAsync(dballs.p, host_balls.data(), sizeof(DevBall) * (k1 - k0), cudaMemcpyHostToDevice, s));
    OM_CUDA(cudaMemsetAsync(dcnt.p, 0, sizeof(unsigned long long) * (k1 - k0), s));
    raster_balls<<<k1 - k0, 256, 0, s>>>(dballs.p, k0, d.nx, d.ny, d.nz, owner.p);
    count_first_cover<<<1216, 256, 0, s>>>(owner.p, N, k0, k1, dcnt.p);
    OM_CUDA(cudaGetLastError());
    cnt.resize(k1 - k0);
    OM_CUDA(cudaMemcpyAsync(cnt.data(), dcnt.p, sizeof(unsigned long long) * (k1 - k0), cudaMemcpyDeviceToHost, s));
    OM_CUDA(cudaStreamSynchronize(s));
    for (int k = k0; k < k1; ++k) {
      covered += (int64_t)cnt[k - k0];
      if ((double)covered / (double)N >= p.porosity) {
        kstop = k;
        break;
      }
    }
  }
  const int klast = kstop >= 0 ? kstop : (int)pl.balls.size() - 1;
  owner_to_mask<<<1216, 256, 0, s>>>(owner.p, N, klast, mask_dev);
  OM_CUDA(cudaGetLastError());
  OM_CUDA(cudaStreamSynchronize(s));
  if (eps_out) *eps_out = (double)covered / (double)N;
  if (nsph_out) *nsph_out = klast + 1;
  if (kstop < 0)
    return fail(OM_EINFEASIBLE, "reconstruction: trial cap reached before the target porosity");
  return OM_OK;
}

}  // namespace
}  // namespace om

using namespace om;

extern "C" om_status om_reconstruct_dev(uint64_t seed, om_domain d, const om_recon_params* params,
                                        uint8_t* mask_dev, double* porosity_out, int64_t* n_spheres_out,
                                        void* stream) {
  if (!params || !mask_dev) return fail(OM_EINVAL, "om_reconstruct_dev: null pointer");
  return reconstruct_impl(seed, d, *params, mask_dev, porosity_out, n_spheres_out, as_stream(stream));
}

extern "C" om_status om_reconstruct(uint64_t seed, om_domain d, const om_recon_params* params,
                                    uint8_t* mask, double* porosity_out, int64_t* n_spheres_out) {
  if (!params || !mask) return fail(OM_EINVAL, "om_reconstruct: null pointer");
  OM_TRY(check_domain(d));
  cudaStream_t s;
  OM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  DevBuf<uint8_t> m;
  om_status st = m.alloc(voxels(d));
  if (st == OM_OK) st = reconstruct_impl(seed, d, *params, m.p, porosity_out, n_spheres_out, s);
  if (st == OM_OK || st == OM_EINFEASIBLE) {
    cudaError_t e = cudaMemcpyAsync(mask, m.p, voxels(d), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "om_reconstruct copy-out", __FILE__, __LINE__);
  }
  cudaStreamDestroy(s);
  return st;
}
