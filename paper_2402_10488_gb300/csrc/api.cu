// Library-level entry points: errors, discretisation (quadrature, distinct sweep directions),
// batches of parametric instances and their parameters.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace rte {

std::atomic<long long> g_launches{0};
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

// Gauss-Legendre nodes on [-1,1] (ascending) with weights normalised to sum 1 (Sec. 2.1):
// Newton iterations on P_n from the recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) {
        p1 = z;
        p0 = 1.0;
      }
      dp = n * (p0 - z * p1) / (1.0 - z * z);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {  // final derivative at the converged node
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0, p1 = z;
      dp = n * (p0 - z * p1) / (1.0 - z * z);
    }
    x[i] = z;
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // textbook 2/(...) times 1/2
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) xs[i] = x[idx[i]], ws[i] = w[idx[i]];
  x.swap(xs);
  w.swap(ws);
}

}  // namespace rte

using namespace rte;

extern "C" int rte_version(void) { return 10900; }
extern "C" const char* rte_last_error(void) { return g_last_error.c_str(); }

extern "C" int rte_disc_create(const rte_disc_desc* d, int device, rte_disc_t* out) {
  if (!d || !out) return fail(RTE_EINVAL, "rte_disc_create: null argument");
  *out = nullptr;
  if (d->dim != 1 && d->dim != 2) return fail(RTE_EINVAL, "dim must be 1 or 2");
  if (d->nx < 1 || d->ny < 1 || (d->dim == 1 && d->ny != 1))
    return fail(RTE_EINVAL, "bad mesh size");
  if (!(d->x1 > d->x0) || (d->dim == 2 && !(d->y1 > d->y0)))
    return fail(RTE_EINVAL, "empty domain");
  if (d->n_mat < 1 || !d->mat_id) return fail(RTE_EINVAL, "need n_mat >= 1 and a material map");
  if (d->dim == 1 && (d->n_phi < 2 || d->n_phi % 2))
    return fail(RTE_EINVAL, "1D: n_phi (GL points) must be even and >= 2");
  if (d->dim == 2 && (d->n_phi < 2 || d->n_phi % 2 || d->n_vz < 1))
    return fail(RTE_EINVAL, "2D: CL(n_phi, n_vz) needs even n_phi >= 2 and n_vz >= 1");
  if ((long long)d->nx * d->ny > (1LL << 28)) return fail(RTE_EINVAL, "mesh too large");
  if (d->dim == 1 && d->dx) {
    double tot = 0.0;
    for (int c = 0; c < d->nx; ++c) {
      if (!std::isfinite(d->dx[c]) || !(d->dx[c] > 0)) return fail(RTE_EINVAL, "cell widths must be positive");
      tot += d->dx[c];
    }
    if (std::fabs(tot - (d->x1 - d->x0)) > 1e-12 * (d->x1 - d->x0))
      return fail(RTE_EINVAL, "cell widths must sum to x1 - x0");
  }
  if (d->mat_id_right) {
    if (d->dim != 1) return fail(RTE_EINVAL, "mat_id_right (linear cross sections) is 1D only");
    for (int c = 0; c < d->nx; ++c)
      if (d->mat_id_right[c] < 0 || d->mat_id_right[c] >= d->n_mat)
        return fail(RTE_EINVAL, "material id out of range");
  }
  int ndev = 0;
  RTE_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(RTE_EINVAL, "bad device index");
  DeviceGuard g(device);

  auto* disc = new rte_disc_s();
  disc->device = device;
  disc->dim = d->dim;
  disc->nx = d->nx;
  disc->ny = d->ny;
  disc->n_cells = d->nx * d->ny;
  disc->P = d->dim == 1 ? 2 : 4;
  disc->n_dof = disc->n_cells * disc->P;
  disc->x0 = d->x0, disc->x1 = d->x1, disc->y0 = d->y0, disc->y1 = d->y1;
  disc->hx = (d->x1 - d->x0) / d->nx;
  if (d->dim == 1) {
    if (d->dx) disc->dx.assign(d->dx, d->dx + d->nx);
    else disc->dx.assign(d->nx, disc->hx);
  }
  disc->hy = d->dim == 2 ? (d->y1 - d->y0) / d->ny : 1.0;
  disc->n_phi = d->n_phi;
  disc->n_vz = d->n_vz;
  disc->n_mat = d->n_mat;
  disc->mat_host.assign(d->mat_id, d->mat_id + disc->n_cells);
  for (int c = 0; c < disc->n_cells; ++c)
    if (disc->mat_host[c] < 0 || disc->mat_host[c] >= d->n_mat) {
      delete disc;
      return fail(RTE_EINVAL, "material id out of range");
    }
  if (d->dim == 1) {
    disc->matr_host = d->mat_id_right ? std::vector<int32_t>(d->mat_id_right, d->mat_id_right + d->nx)
                                      : disc->mat_host;
    disc->linear = disc->matr_host != disc->mat_host;
  }

  // ---- quadrature (Sec. 2.1) and distinct directions --------------------------------------
  if (d->dim == 1) {
    std::vector<double> x, w;
    gauss_legendre(d->n_phi, x, w);
    disc->n_angles = d->n_phi;
    disc->v.assign(3 * d->n_phi, 0.0);
    disc->w = w;
    for (int j = 0; j < d->n_phi; ++j) {
      disc->v[3 * j] = x[j];
      Dir dd{x[j], 0.0, w[j], 1, x[j] < 0 ? 1 : 0};
      disc->dirs.push_back(dd);
    }
  } else {
    std::vector<double> vz, wz;
    gauss_legendre(d->n_vz, vz, wz);
    const int np = d->n_phi, nz = d->n_vz;
    disc->n_angles = np * nz;
    disc->v.assign(3 * np * nz, 0.0);
    disc->w.assign(np * nz, 0.0);
    for (int j2 = 0; j2 < nz; ++j2) {
      double s = std::sqrt(1.0 - vz[j2] * vz[j2]);
      for (int j1 = 0; j1 < np; ++j1) {
        double phi = 2.0 * (j1 + 1) * M_PI / np - M_PI / np;
        int j = j2 * np + j1;
        disc->v[3 * j] = std::cos(phi) * s;
        disc->v[3 * j + 1] = std::sin(phi) * s;
        disc->v[3 * j + 2] = vz[j2];
        disc->w[j] = (1.0 / np) * wz[j2];
      }
    }
    // GL in v_z is symmetric: level j2 and nz-1-j2 carry the same (v_x, v_y) and weight, so
    // their transport solutions coincide; sweep each pair once with the summed weight.
    for (int j2 = 0; j2 < (nz + 1) / 2; ++j2) {
      int mirror = nz - 1 - j2;
      int mult = mirror == j2 ? 1 : 2;
      for (int j1 = 0; j1 < np; ++j1) {
        int j = j2 * np + j1;
        double vx = disc->v[3 * j], vy = disc->v[3 * j + 1];
        double w = disc->w[j] + (mult == 2 ? disc->w[mirror * np + j1] : 0.0);
        disc->dirs.push_back(Dir{vx, vy, w, mult, (vx < 0 ? 1 : 0) + (vy < 0 ? 2 : 0)});
      }
    }
  }
  std::stable_sort(disc->dirs.begin(), disc->dirs.end(),
                   [](const Dir& a, const Dir& b) { return a.quad < b.quad; });
  disc->n_dirs = (int)disc->dirs.size();

  // DSA moments over the full rule (App. B)
  {
    DsaMoments m{};
    for (int j = 0; j < disc->n_angles; ++j) {
      double vx = disc->v[3 * j], vy = disc->v[3 * j + 1], w = disc->w[j];
      m.abs_x += w * std::fabs(vx);
      m.abs_y += w * std::fabs(vy);
      m.xx += w * vx * vx;
      m.yy += w * vy * vy;
      m.abs3_x += w * std::fabs(vx) * vx * vx;
      m.abs3_y += w * std::fabs(vy) * vy * vy;
      m.xx_absy += w * vx * vx * std::fabs(vy);
      m.yy_absx += w * vy * vy * std::fabs(vx);
    }
    disc->mom = m;
  }

  int st = disc->mat_id.alloc(disc->n_cells);
  if (st == RTE_OK) st = disc->dir_dev.alloc(4 * (size_t)disc->n_dirs);
  if (st == RTE_OK && d->dim == 1) st = disc->dx_dev.alloc(disc->nx);
  if (st == RTE_OK && disc->linear) st = disc->mat_r.alloc(disc->nx);
  if (st != RTE_OK) {
    delete disc;
    return st;
  }
  std::vector<double> dh(4 * disc->n_dirs);
  for (int k = 0; k < disc->n_dirs; ++k) {
    dh[4 * k] = disc->dirs[k].vx;
    dh[4 * k + 1] = disc->dirs[k].vy;
    dh[4 * k + 2] = disc->dirs[k].w;
    dh[4 * k + 3] = disc->dirs[k].mult;
  }
  cudaError_t e1 = cudaMemcpy(disc->mat_id.p, disc->mat_host.data(),
                              sizeof(int32_t) * disc->n_cells, cudaMemcpyHostToDevice);
  cudaError_t e2 =
      cudaMemcpy(disc->dir_dev.p, dh.data(), sizeof(double) * dh.size(), cudaMemcpyHostToDevice);
  cudaError_t e3 = cudaSuccess;
  if (d->dim == 1)
    e3 = cudaMemcpy(disc->dx_dev.p, disc->dx.data(), sizeof(double) * disc->nx, cudaMemcpyHostToDevice);
  if (e3 == cudaSuccess && disc->linear)
    e3 = cudaMemcpy(disc->mat_r.p, disc->matr_host.data(), sizeof(int32_t) * disc->nx,
                    cudaMemcpyHostToDevice);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    delete disc;
    return fail(RTE_ECUDA, "rte_disc_create: upload failed");
  }
  *out = disc;
  return RTE_OK;
}

extern "C" int rte_disc_destroy(rte_disc_t disc) {
  if (!disc) return RTE_OK;
  DeviceGuard g(disc->device);
  delete disc;
  return RTE_OK;
}

extern "C" int rte_disc_info(rte_disc_t disc, int64_t* info) {
  if (!disc || !info) return fail(RTE_EINVAL, "rte_disc_info: null argument");
  info[0] = disc->n_cells;
  info[1] = disc->n_dof;
  info[2] = disc->P;
  info[3] = disc->n_angles;
  info[4] = disc->n_dirs;
  info[5] = disc->n_mat;
  info[6] = disc->dim;
  info[7] = disc->device;
  return RTE_OK;
}

extern "C" int rte_disc_quadrature(rte_disc_t disc, double* v, double* omega) {
  if (!disc || !v || !omega) return fail(RTE_EINVAL, "rte_disc_quadrature: null argument");
  std::memcpy(v, disc->v.data(), sizeof(double) * disc->v.size());
  std::memcpy(omega, disc->w.data(), sizeof(double) * disc->w.size());
  return RTE_OK;
}

// ---- batches ------------------------------------------------------------------------------

namespace rte {
// sweep work groups: per quadrant, consecutive runs of <= dpw directions
void make_groups(rte_batch_t b) {
  const rte_disc_s* disc = b->disc;
  b->groups.clear();
  int d = 0;
  while (d < disc->n_dirs) {
    const int q = disc->dirs[d].quad;
    int e = d;
    while (e < disc->n_dirs && disc->dirs[e].quad == q && e - d < b->dpw) ++e;
    b->groups.push_back(SweepGroup{d, e - d, q, 0});
    d = e;
  }
}

static std::vector<SweepGroup> groups_for(const rte_disc_s* disc, int dpw) {
  std::vector<SweepGroup> g;
  int d = 0;
  while (d < disc->n_dirs) {
    const int q = disc->dirs[d].quad;
    int e = d;
    while (e < disc->n_dirs && disc->dirs[e].quad == q && e - d < dpw) ++e;
    g.push_back(SweepGroup{d, e - d, q, 0});
    d = e;
  }
  return g;
}

void pick_groups(rte_batch_t b, int n_active, int* dpw, int* n_groups, const SweepGroup** dev,
                 bool f32) {
  int use = b->dpw;
  auto kof = [](int v) { return v == 1 ? 0 : v == 2 ? 1 : v == 4 ? 2 : 3; };
  const auto& tuned = f32 && !b->tuned32.empty() ? b->tuned32 : b->tuned;
  if (b->force_dpw && b->disc->dim == 2) {
    use = b->force_dpw;
  } else if (b->dpw_dynamic && b->disc->dim == 2) {
    if (!tuned.empty()) {
      use = tuned.back().second;
      for (const auto& e : tuned)
        if (n_active <= e.first) {
          use = e.second;
          break;
        }
    } else {
      use = 1;
      for (int k = 3; k >= 1; --k) {
        const int cand = 1 << k;
        if (cand > b->dpw) continue;
        if ((long long)n_active * b->gcount[k] >= 4LL * b->n_sm) {
          use = cand;
          break;
        }
      }
    }
    // partial sums are indexed by the rank among running instances: a finer decomposition fits
    // when few instances run; otherwise widen the groups until the buffer holds them
    const size_t cap = b->partial.n / std::max(b->disc->n_dof, 1);
    while (use < kMaxDirsPerWarp && (size_t)std::max(n_active, 1) * b->gcount[kof(use)] > cap) use *= 2;
  }
  const int k = kof(use);
  if (b->disc->dim == 2 && b->groups_all_dev.p) {
    *dpw = use;
    *n_groups = b->gcount[k];
    *dev = b->groups_all_dev.p + b->goff[k];
  } else {
    *dpw = b->dpw;
    *n_groups = (int)b->groups.size();
    *dev = b->groups_dev.p;
  }
}

// largest directions-per-warp giving >= 4 resident warps per SM (each SM sub-partition has its
// own FP64 unit, so one warp per sub-partition is the minimum to use the SM's FP64 rate)
int auto_dpw(const rte_disc_s* disc, int B) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, disc->device) != cudaSuccess || sms < 1)
    sms = 148;
  int per_quad[4] = {0, 0, 0, 0};
  for (const auto& d : disc->dirs) per_quad[d.quad]++;
  for (int dpw : {8, 4, 2}) {
    long long warps = 0;
    for (int q = 0; q < 4; ++q) warps += (long long)B * ((per_quad[q] + dpw - 1) / dpw);
    if (warps >= 4LL * sms) return dpw;
  }
  return 1;
}
}  // namespace rte

extern "C" int rte_batch_tune(rte_batch_t b, int dpw) {
  if (!b) return fail(RTE_EINVAL, "rte_batch_tune: null argument");
  if (b->disc->dim == 1) return RTE_OK;
  b->dpw_dynamic = dpw == 0;
  b->tuned.clear();
  b->tuned32.clear();
  b->tuned_nw.clear();
  if (dpw == 0) dpw = std::max(auto_dpw(b->disc, b->B), b->min_dpw);
  if (dpw != 1 && dpw != 2 && dpw != 4 && dpw != 8) return fail(RTE_EINVAL, "dirs_per_warp must be 0, 1, 2, 4 or 8");
  DeviceGuard g(b->disc->device);
  const int old = b->dpw;
  b->dpw = dpw;
  make_groups(b);
  const size_t need = (size_t)b->B * b->groups.size() * b->disc->n_dof;
  if (need > b->partial.n) {
    int st = b->partial.alloc(need);
    if (st != RTE_OK) {
      b->dpw = old;
      make_groups(b);
      b->partial.alloc((size_t)b->B * b->groups.size() * b->disc->n_dof);
      return st;
    }
  }
  RTE_TRY(b->groups_dev.alloc(b->groups.size()));
  RTE_CUDA_TRY(cudaMemcpy(b->groups_dev.p, b->groups.data(), sizeof(SweepGroup) * b->groups.size(),
                          cudaMemcpyHostToDevice));
  return RTE_OK;
}

size_t rte_batch_s::bytes() const {
  size_t t = 8 * (sigma_t.n + sigma_s.n + G0.n + inflow.n + tables.n + partial.n + S.n + norms.n + work.n +
                  outer.n + leak.n + vout.n);
  t += 4 * (tables32.n + S32.n + partial32.n + tablesff.n + Sff.n);
  t += sizeof(rte::SweepGroup) * (groups_dev.n + groups_all_dev.n) + slot_mask.n;
  return t + rte::dsa_bytes(this);
}

rte_batch_s::~rte_batch_s() {
  if (param_bad_h) cudaFreeHost(param_bad_h);
  if (param_ev) cudaEventDestroy(param_ev);
  if (stage) cudaFreeHost(stage);
  if (stage_mask) cudaFreeHost(stage_mask);
  if (stage_ev) cudaEventDestroy(stage_ev);
  rte::dsa_state_free(dsa);
  for (auto& e : sweep_ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : phase_ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
}

extern "C" int rte_counters(int64_t* out) {
  if (!out) return fail(RTE_EINVAL, "rte_counters: null argument");
  out[0] = rte::g_launches.load();
  return RTE_OK;
}

extern "C" int rte_batch_timing(rte_batch_t b, int enable, double* out) {
  if (!b) return fail(RTE_EINVAL, "rte_batch_timing: null argument");
  DeviceGuard g(b->disc->device);
  double ms = 0.0, pms[5] = {0, 0, 0, 0, 0};
  for (auto& e : b->sweep_ev) {
    RTE_CUDA_TRY(cudaEventSynchronize(e.second));
    float t = 0.f;
    RTE_CUDA_TRY(cudaEventElapsedTime(&t, e.first, e.second));
    ms += t;
  }
  for (auto& e : b->phase_ev) {
    RTE_CUDA_TRY(cudaEventSynchronize(e.b));
    float t = 0.f;
    RTE_CUDA_TRY(cudaEventElapsedTime(&t, e.a, e.b));
    pms[e.phase] += t;
  }
  if (out) {
    out[0] = ms;
    out[1] = (double)b->sweep_launches;
    out[2] = b->sweep_units;
    for (int p = 1; p <= 3; ++p) {
      out[1 + 2 * p] = pms[p];
      out[2 + 2 * p] = (double)b->phase_calls[p];
    }
    out[9] = pms[0];
    out[10] = (double)b->phase_calls[0];
    out[11] = b->sweep32_units;
    out[12] = pms[4];
    out[13] = (double)b->phase_calls[4];
    out[14] = b->sweepff_units;
  }
  if (enable >= 0) {
    for (auto& e : b->sweep_ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    for (auto& e : b->phase_ev) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    b->sweep_ev.clear();
    b->phase_ev.clear();
    for (auto& c : b->phase_calls) c = 0;
    b->sweep_units = 0.0;
    b->sweep32_units = 0.0;
    b->sweepff_units = 0.0;
    b->sweep_launches = 0;
    b->timing = enable != 0;
  }
  return RTE_OK;
}

extern "C" int rte_batch_create(rte_disc_t disc, int B, rte_batch_t* out) {
  if (!disc || !out || B < 1) return fail(RTE_EINVAL, "rte_batch_create: bad argument");
  *out = nullptr;
  DeviceGuard g(disc->device);
  auto* b = new rte_batch_s();
  b->disc = disc;
  b->B = B;
  std::vector<SweepGroup> all;
  if (disc->dim == 2) {
    if (cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, disc->device) != cudaSuccess)
      b->n_sm = 148;
    for (int k = 0; k < 4; ++k) {
      auto g = groups_for(disc, 1 << k);
      b->goff[k] = (int)all.size();
      b->gcount[k] = (int)g.size();
      all.insert(all.end(), g.begin(), g.end());
    }
    // per-instance partial sums stay within kPartialBytes: large discretisations use wider groups
    int k = 0;
    while (k < 3 && (size_t)b->gcount[k] * disc->n_dof * sizeof(double) > kPartialBytes) ++k;
    b->min_dpw = 1 << k;
  }
  b->dpw = disc->dim == 1 ? 1 : std::max(auto_dpw(disc, B), b->min_dpw);
  make_groups(b);
  const size_t max_groups =
      disc->dim == 2 ? (size_t)b->gcount[b->min_dpw == 1 ? 0 : b->min_dpw == 2 ? 1 : b->min_dpw == 4 ? 2 : 3]
                     : b->groups.size();
  const size_t nb = (size_t)B;
  const size_t tab = disc->dim == 1 ? kTab1D : kTab2D;
  int st = RTE_OK;
  if (st == RTE_OK) st = b->groups_dev.alloc(b->groups.size());
  if (st == RTE_OK) st = b->sigma_t.alloc(nb * disc->n_mat);
  if (st == RTE_OK) st = b->sigma_s.alloc(nb * disc->n_mat);
  if (st == RTE_OK) st = b->G0.alloc(nb * disc->n_cells);
  if (st == RTE_OK) st = b->inflow.alloc(nb * 4);
  // sweep tables per (instance, material, direction) in 2D; per (instance, cell, direction) in 1D
  // (the cell width enters the table and 1D meshes may be non-uniform)
  const size_t tab_units = disc->dim == 1 ? (size_t)disc->n_cells : (size_t)disc->n_mat;
  if (st == RTE_OK) st = b->tables.alloc(nb * tab_units * disc->n_dirs * tab);
  if (st == RTE_OK) st = b->partial.alloc(nb * max_groups * disc->n_dof);
  if (st == RTE_OK && !all.empty()) st = b->groups_all_dev.alloc(all.size());
  if (st == RTE_OK) st = b->norms.alloc(nb * 2);
  if (st == RTE_OK && disc->dim == 2) st = b->S.alloc(nb * disc->n_dof);
  if (st == RTE_OK) st = b->work.alloc(nb * disc->n_dof * 4);
  // the allocation-free sweep's static scratch is loaded on this device now, at set-up, so that
  // rte_sweep_static itself never triggers the load (and its allocation)
  if (st == RTE_OK) st = rte::static_scratch_preload();
  if (st != RTE_OK) {
    delete b;
    return st;
  }
  if ((!all.empty() && cudaMemcpy(b->groups_all_dev.p, all.data(), sizeof(SweepGroup) * all.size(),
                                  cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(b->groups_dev.p, b->groups.data(), sizeof(SweepGroup) * b->groups.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    delete b;
    return fail(RTE_ECUDA, "rte_batch_create: upload failed");
  }
  *out = b;
  return RTE_OK;
}

extern "C" int rte_batch_destroy(rte_batch_t b) {
  if (!b) return RTE_OK;
  DeviceGuard g(b->disc->device);
  delete b;
  return RTE_OK;
}

namespace rte {
// Parameters from device memory: the cross-section tables copied, G0 = G sqrt|T| per cell (the
// zeroth moment of a cellwise-constant source on the orthonormal basis, as the host path computes
// it), the inflow spread to the [B][4] layout, and `bad` set when a value is not finite or
// violates sigma_t > 0, 0 <= sigma_s <= sigma_t.  Grid-stride over the largest of the three.
__global__ void params_device_kernel(const double* __restrict__ sigma_t,
                                     const double* __restrict__ sigma_s,
                                     const double* __restrict__ source,
                                     const double* __restrict__ inflow, double* st_out,
                                     double* ss_out, double* G0, double* inflow_out,
                                     const double* __restrict__ dx, double sq_area, int B,
                                     int n_mat, int n_cells, int n_side, int* bad) {
  const size_t nm = (size_t)B * n_mat, nc = (size_t)B * n_cells, ni = (size_t)B * 4;
  const size_t n = nm > nc ? (nm > ni ? nm : ni) : (nc > ni ? nc : ni);
  bool ok = true;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    if (k < nm) {
      const double t = sigma_t[k], c = sigma_s[k];
      ok = ok && isfinite(t) && isfinite(c) && t > 0.0 && c >= 0.0 && c <= t;
      st_out[k] = t;
      ss_out[k] = c;
    }
    if (k < nc) {
      const double g = source[k];
      ok = ok && isfinite(g);
      G0[k] = g * (dx ? sqrt(dx[k % n_cells]) : sq_area);
    }
    if (k < ni) {
      const int side = (int)(k % 4);
      const double g = side < n_side ? inflow[(k / 4) * n_side + side] : 0.0;
      ok = ok && isfinite(g);
      inflow_out[k] = g;
    }
  }
  if (!ok) atomicOr(bad, 1);
}

int params_ready(rte_batch_t b, const char* who) {
  if (b->param_pending) {
    RTE_CUDA_TRY(cudaEventSynchronize(b->param_ev));
    b->param_pending = false;
    if (*b->param_bad_h) {
      b->params_set = false;
      return fail(RTE_EINVAL, std::string(who) + ": the parameters set from device memory are "
                  "invalid (need finite values, sigma_t > 0 and 0 <= sigma_s <= sigma_t)");
    }
  }
  if (!b->params_set) return fail(RTE_ESTATE, std::string(who) + ": parameters not set");
  return RTE_OK;
}
}  // namespace rte

extern "C" int rte_batch_set_params_device(rte_batch_t b, const double* sigma_t,
                                           const double* sigma_s, const double* source,
                                           const double* inflow, void* stream) {
  if (!b || !sigma_t || !sigma_s || !source || !inflow)
    return fail(RTE_EINVAL, "rte_batch_set_params_device: null argument");
  rte_disc_s* d = b->disc;
  DeviceGuard g(d->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (b->param_pending) {       // a previous device upload's flag must be read before reuse
    RTE_CUDA_TRY(cudaEventSynchronize(b->param_ev));
    b->param_pending = false;
  }
  if (!b->param_bad.p) {
    RTE_TRY(b->param_bad.alloc(1));
    RTE_CUDA_TRY(cudaHostAlloc((void**)&b->param_bad_h, sizeof(int), cudaHostAllocDefault));
    RTE_CUDA_TRY(cudaEventCreateWithFlags(&b->param_ev, cudaEventDisableTiming));
  }
  const size_t nm = (size_t)b->B * d->n_mat, nc = (size_t)b->B * d->n_cells;
  const size_t n = std::max(std::max(nm, nc), (size_t)b->B * 4);
  RTE_CUDA_TRY(cudaMemsetAsync(b->param_bad.p, 0, sizeof(int), st));
  const int th = 256;
  const unsigned bl = (unsigned)std::min<size_t>((n + th - 1) / th, 4096);
  params_device_kernel<<<bl, th, 0, st>>>(sigma_t, sigma_s, source, inflow, b->sigma_t.p,
                                          b->sigma_s.p, b->G0.p, b->inflow.p,
                                          d->dim == 1 ? d->dx_dev.p : nullptr,
                                          std::sqrt(d->hx * d->hy), b->B, d->n_mat, d->n_cells,
                                          2 * d->dim, b->param_bad.p); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  {
    PhaseScope ps(b, 3, st);
    RTE_TRY(setup_tables(b, st));
    b->tables32_stale = true;
    b->tablesff_stale = true;
    RTE_TRY(dsa_setup(b, st));
  }
  RTE_CUDA_TRY(cudaMemcpyAsync(b->param_bad_h, b->param_bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  RTE_CUDA_TRY(cudaEventRecord(b->param_ev, st));
  b->param_pending = true;
  b->slot_set.assign(b->B, 1);
  b->params_set = true;
  return RTE_OK;
}

extern "C" int rte_batch_set_params(rte_batch_t b, const double* sigma_t, const double* sigma_s,
                                    const double* source, const double* inflow) {
  if (!b || !sigma_t || !sigma_s || !source || !inflow)
    return fail(RTE_EINVAL, "rte_batch_set_params: null argument");
  rte_disc_s* d = b->disc;
  const size_t nm = (size_t)b->B * d->n_mat, nc = (size_t)b->B * d->n_cells;
  const size_t ni = (size_t)b->B * 2 * d->dim;
  for (size_t k = 0; k < nm; ++k) {
    if (!std::isfinite(sigma_t[k]) || !std::isfinite(sigma_s[k]))
      return fail(RTE_EINVAL, "cross section is not finite");
    if (!(sigma_t[k] > 0.0) || sigma_s[k] < 0.0 || sigma_s[k] > sigma_t[k])
      return fail(RTE_EINVAL, "need sigma_t > 0 and 0 <= sigma_s <= sigma_t");
  }
  for (size_t k = 0; k < nc; ++k)
    if (!std::isfinite(source[k])) return fail(RTE_EINVAL, "source is not finite");
  for (size_t k = 0; k < ni; ++k)
    if (!std::isfinite(inflow[k])) return fail(RTE_EINVAL, "inflow is not finite");
  DeviceGuard g(d->device);
  if (b->param_pending) {       // a device upload still in flight is superseded by this one
    RTE_CUDA_TRY(cudaEventSynchronize(b->param_ev));
    b->param_pending = false;
  }
  b->sigma_t_h.assign(sigma_t, sigma_t + nm);
  b->sigma_s_h.assign(sigma_s, sigma_s + nm);
  b->source_h.assign(source, source + nc);
  b->inflow_h.assign(4 * (size_t)b->B, 0.0);
  for (int i = 0; i < b->B; ++i)
    for (int s = 0; s < 2 * d->dim; ++s) b->inflow_h[4 * i + s] = inflow[2 * d->dim * i + s];
  // zeroth moment of a cellwise-constant source: int_T G phi_0 = G sqrt(|T|)
  std::vector<double> g0(nc);
  for (size_t k = 0; k < nc; ++k)
    g0[k] = source[k] * (d->dim == 1 ? std::sqrt(d->dx[k % d->n_cells]) : std::sqrt(d->hx * d->hy));
  RTE_CUDA_TRY(cudaMemcpy(b->sigma_t.p, sigma_t, sizeof(double) * nm, cudaMemcpyHostToDevice));
  RTE_CUDA_TRY(cudaMemcpy(b->sigma_s.p, sigma_s, sizeof(double) * nm, cudaMemcpyHostToDevice));
  RTE_CUDA_TRY(cudaMemcpy(b->G0.p, g0.data(), sizeof(double) * nc, cudaMemcpyHostToDevice));
  RTE_CUDA_TRY(cudaMemcpy(b->inflow.p, b->inflow_h.data(), sizeof(double) * 4 * b->B,
                          cudaMemcpyHostToDevice));
  {
    PhaseScope ps(b, 3, 0);
    RTE_TRY(setup_tables(b, 0));
    b->tables32_stale = true;
    b->tablesff_stale = true;
    RTE_TRY(dsa_setup(b, 0));
  }
  RTE_CUDA_TRY(cudaDeviceSynchronize());
  b->slot_set.assign(b->B, 1);
  b->params_set = true;
  return RTE_OK;
}

namespace rte {
int set_slots(rte_batch_t b, int n, const int* slots, const double* sigma_t, const double* sigma_s,
              const double* source, const double* inflow, cudaStream_t st) {
  rte_disc_s* d = b->disc;
  const int B = b->B, nm = d->n_mat, nc = d->n_cells, ni = 2 * d->dim;
  const size_t per = 2 * (size_t)nm + nc + 4;
  for (int i = 0; i < n; ++i) {
    if (slots[i] < 0 || slots[i] >= B) return fail(RTE_EINVAL, "slot out of range");
    for (int j = 0; j < i; ++j)
      if (slots[j] == slots[i]) return fail(RTE_EINVAL, "slot listed twice");
  }
  for (size_t k = 0; k < (size_t)n * nm; ++k) {
    if (!std::isfinite(sigma_t[k]) || !std::isfinite(sigma_s[k]))
      return fail(RTE_EINVAL, "cross section is not finite");
    if (!(sigma_t[k] > 0.0) || sigma_s[k] < 0.0 || sigma_s[k] > sigma_t[k])
      return fail(RTE_EINVAL, "need sigma_t > 0 and 0 <= sigma_s <= sigma_t");
  }
  for (size_t k = 0; k < (size_t)n * nc; ++k)
    if (!std::isfinite(source[k])) return fail(RTE_EINVAL, "source is not finite");
  for (size_t k = 0; k < (size_t)n * ni; ++k)
    if (!std::isfinite(inflow[k])) return fail(RTE_EINVAL, "inflow is not finite");
  if (!b->stage) {
    RTE_CUDA_TRY(cudaHostAlloc((void**)&b->stage, sizeof(double) * per * B, cudaHostAllocDefault));
    RTE_CUDA_TRY(cudaHostAlloc((void**)&b->stage_mask, B, cudaHostAllocDefault));
    RTE_CUDA_TRY(cudaEventCreateWithFlags(&b->stage_ev, cudaEventDisableTiming));
    RTE_TRY(b->slot_mask.alloc(B));
  } else {
    RTE_CUDA_TRY(cudaEventSynchronize(b->stage_ev));  // the previous upload has been consumed
  }
  if (b->sigma_t_h.size() != (size_t)B * nm) {
    b->sigma_t_h.assign((size_t)B * nm, 1.0);
    b->sigma_s_h.assign((size_t)B * nm, 0.0);
    b->source_h.assign((size_t)B * nc, 0.0);
    b->inflow_h.assign(4 * (size_t)B, 0.0);
  }
  if (b->slot_set.size() != (size_t)B) b->slot_set.assign(B, 0);
  std::memset(b->stage_mask, 0, B);
  for (int i = 0; i < n; ++i) {
    const int sl = slots[i];
    double* p = b->stage + per * sl;
    for (int m = 0; m < nm; ++m) {
      p[m] = b->sigma_t_h[(size_t)sl * nm + m] = sigma_t[(size_t)i * nm + m];
      p[nm + m] = b->sigma_s_h[(size_t)sl * nm + m] = sigma_s[(size_t)i * nm + m];
    }
    for (int c = 0; c < nc; ++c) {
      b->source_h[(size_t)sl * nc + c] = source[(size_t)i * nc + c];
      p[2 * nm + c] = source[(size_t)i * nc + c] *   // zeroth moment of the cell source
                      (d->dim == 1 ? std::sqrt(d->dx[c]) : std::sqrt(d->hx * d->hy));
    }
    for (int k = 0; k < 4; ++k)
      p[2 * nm + nc + k] = b->inflow_h[4 * (size_t)sl + k] = k < ni ? inflow[(size_t)i * ni + k] : 0.0;
    b->stage_mask[sl] = 1;
    b->slot_set[sl] = 1;
    RTE_CUDA_TRY(cudaMemcpyAsync(b->sigma_t.p + (size_t)sl * nm, p, sizeof(double) * nm, cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaMemcpyAsync(b->sigma_s.p + (size_t)sl * nm, p + nm, sizeof(double) * nm, cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaMemcpyAsync(b->G0.p + (size_t)sl * nc, p + 2 * nm, sizeof(double) * nc, cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaMemcpyAsync(b->inflow.p + 4 * (size_t)sl, p + 2 * nm + nc, sizeof(double) * 4, cudaMemcpyHostToDevice, st));
  }
  RTE_CUDA_TRY(cudaMemcpyAsync(b->slot_mask.p, b->stage_mask, B, cudaMemcpyHostToDevice, st));
  {
    PhaseScope ps(b, 3, st);
    RTE_TRY(setup_tables(b, st, b->slot_mask.p));
    b->tables32_stale = true;
    b->tablesff_stale = true;
    RTE_TRY(dsa_setup(b, st, b->slot_mask.p));
  }
  RTE_CUDA_TRY(cudaEventRecord(b->stage_ev, st));
  bool all = true;
  for (int k = 0; k < B; ++k) all = all && b->slot_set[k];
  if (all) b->params_set = true;
  return RTE_OK;
}
}  // namespace rte

extern "C" int rte_batch_set_slots(rte_batch_t b, int n, const int* slots, const double* sigma_t,
                                   const double* sigma_s, const double* source,
                                   const double* inflow, void* stream) {
  if (!b || n < 0 || (n > 0 && (!slots || !sigma_t || !sigma_s || !source || !inflow)))
    return fail(RTE_EINVAL, "rte_batch_set_slots: null argument");
  if (n == 0) return RTE_OK;
  DeviceGuard g(b->disc->device);
  return set_slots(b, n, slots, sigma_t, sigma_s, source, inflow, (cudaStream_t)stream);
}

extern "C" int rte_batch_info(rte_batch_t b, int64_t* info) {
  if (!b || !info) return fail(RTE_EINVAL, "rte_batch_info: null argument");
  info[0] = b->B;
  info[1] = (int64_t)b->bytes();
  info[2] = b->dpw;
  info[3] = b->min_dpw;
  info[4] = b->dpw_dynamic ? 1 : 0;
  info[5] = b->params_set ? 1 : 0;
  return RTE_OK;
}

extern "C" int rte_batch_directions(rte_batch_t b, double* dirs) {
  if (!b || !dirs) return fail(RTE_EINVAL, "rte_batch_directions: null argument");
  const rte_disc_s* d = b->disc;
  for (int k = 0; k < d->n_dirs; ++k) {
    dirs[4 * k] = d->dirs[k].vx;
    dirs[4 * k + 1] = d->dirs[k].vy;
    dirs[4 * k + 2] = d->dirs[k].w;
    dirs[4 * k + 3] = d->dirs[k].mult;
  }
  return RTE_OK;
}
