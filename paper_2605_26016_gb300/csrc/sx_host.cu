// Host side of the library: contexts, distance shells, the coupling table
// (directed taps of the multi-channel convolution kernel K_ab(delta)),
// planning, argument checks and the C-ABI entry points of sx.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "sx_internal.h"

namespace {

thread_local std::string g_err;

}  // namespace

namespace sx {

int set_error(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  return set_error(e == cudaErrorMemoryAllocation ? SX_ERR_OOM : SX_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

int take_status(sx_ctx *c, cudaStream_t st) {
  if (!c->d_status) return SX_OK;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "status read");
  if (!(h & kStatusNumeric)) return SX_OK;
  e = cudaMemsetAsync(c->d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "status reset");
  return set_error(SX_ERR_NUMERIC,
                   "a spin update met a non-finite or zero-length spin since the last check: the state is invalid");
}

namespace {

inline void to_cart(const sx_lattice &L, const double f[3], double r[3]) {
  for (int k = 0; k < 3; ++k) r[k] = f[0] * L.a[0][k] + f[1] * L.a[1][k] + f[2] * L.a[2][k];
}

inline double length(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

// displacement (nm) from sublattice a at cell 0 to sublattice b at cell d
inline void bond_vector(const sx_lattice &L, int a, int b, int dx, int dy, int dz, double r[3]) {
  const double f[3] = {dx + L.sub_pos[b][0] - L.sub_pos[a][0], dy + L.sub_pos[b][1] - L.sub_pos[a][1],
                       dz + L.sub_pos[b][2] - L.sub_pos[a][2]};
  to_cart(L, f, r);
}

double cell_volume(const sx_lattice &L) {
  const double *u = L.a[0], *v = L.a[1], *w = L.a[2];
  return u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) + u[2] * (v[0] * w[1] - v[1] * w[0]);
}

// distance up to which every translation is inside the +-kSearch box
double search_reach(const sx_lattice &L) {
  const double V = fabs(cell_volume(L));
  double h = 1e300;
  for (int k = 0; k < 3; ++k) {
    const double *u = L.a[(k + 1) % 3], *v = L.a[(k + 2) % 3];
    const double c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    h = std::min(h, V / length(c));
  }
  return (kSearch - 1) * h;
}

void compute_shells(sx_ctx *c) {
  std::vector<double> d;
  const sx_lattice &L = c->lat;
  for (int a = 0; a < L.nsub; ++a)
    for (int b = 0; b < L.nsub; ++b)
      for (int dz = -kSearch; dz <= kSearch; ++dz)
        for (int dy = -kSearch; dy <= kSearch; ++dy)
          for (int dx = -kSearch; dx <= kSearch; ++dx) {
            double r[3];
            bond_vector(L, a, b, dx, dy, dz, r);
            const double len = length(r);
            if (len > c->tol) d.push_back(len);
          }
  std::sort(d.begin(), d.end());
  c->nshell = 0;
  for (double v : d) {
    if (c->nshell == 256) break;
    if (c->nshell == 0 || v - c->shell_r[c->nshell - 1] > c->tol) c->shell_r[c->nshell++] = v;
  }
}

int shell_index(const sx_ctx *c, double len) {
  const double *lo = std::lower_bound(c->shell_r, c->shell_r + c->nshell, len - c->tol);
  if (lo == c->shell_r + c->nshell || fabs(*lo - len) > c->tol) return -1;
  return (int)(lo - c->shell_r);
}

// Directed taps per target sublattice from shells, DMI and raw bonds.
void build_tables(sx_ctx *c) {
  const sx_lattice &L = c->lat;
  const int W = 2 * kSearch + 1;
  const int nslot = L.nsub * W * W * W;
  c->taps.assign(L.nsub, {});
  c->radius[0] = c->radius[1] = c->radius[2] = 0;
  for (int a = 0; a < L.nsub; ++a) {
    std::vector<double> acc((size_t)nslot * 9, 0.0);
    std::vector<char> used(nslot, 0);
    auto slot = [&](int b, int dx, int dy, int dz) {
      return ((b * W + (dz + kSearch)) * W + (dy + kSearch)) * W + (dx + kSearch);
    };
    for (int b = 0; b < L.nsub; ++b)
      for (int dz = -kSearch; dz <= kSearch; ++dz)
        for (int dy = -kSearch; dy <= kSearch; ++dy)
          for (int dx = -kSearch; dx <= kSearch; ++dx) {
            double r[3];
            bond_vector(L, a, b, dx, dy, dz, r);
            const double len = length(r);
            if (len <= c->tol) continue;
            const int k = shell_index(c, len);
            if (k < 0 || k >= SX_MAX_SHELL) continue;
            double *J = &acc[(size_t)slot(b, dx, dy, dz) * 9];
            if (c->shellJ[k] != 0.0) {
              J[0] += c->shellJ[k];
              J[4] += c->shellJ[k];
              J[8] += c->shellJ[k];
              used[slot(b, dx, dy, dz)] = 1;
            }
            if (c->dmiD[k] != 0.0) {
              const double e[3] = {r[0] / len, r[1] / len, r[2] / len};
              double D[3];
              bool on = true;
              if (c->dmi_kind[k] == SX_DMI_INTERFACIAL) {
                on = fabs(r[2]) <= c->tol;
                D[0] = -c->dmiD[k] * e[1];
                D[1] = c->dmiD[k] * e[0];
                D[2] = 0.0;
              } else {
                D[0] = c->dmiD[k] * e[0];
                D[1] = c->dmiD[k] * e[1];
                D[2] = c->dmiD[k] * e[2];
              }
              if (on) {
                // J_ij S_j gains S_j x D_ij
                J[1] += D[2];
                J[2] += -D[1];
                J[3] += -D[2];
                J[5] += D[0];
                J[6] += D[1];
                J[7] += -D[0];
                used[slot(b, dx, dy, dz)] = 1;
              }
            }
          }
    for (const sx_bond &o : c->bonds) {
      if (o.a == a) {
        double *J = &acc[(size_t)slot(o.b, o.d[0], o.d[1], o.d[2]) * 9];
        for (int k = 0; k < 9; ++k) J[k] += o.J[k];
        used[slot(o.b, o.d[0], o.d[1], o.d[2])] = 1;
      }
      if (o.b == a) {
        double *J = &acc[(size_t)slot(o.a, -o.d[0], -o.d[1], -o.d[2]) * 9];
        for (int r = 0; r < 3; ++r)
          for (int q = 0; q < 3; ++q) J[3 * r + q] += o.J[3 * q + r];
        used[slot(o.a, -o.d[0], -o.d[1], -o.d[2])] = 1;
      }
    }
    for (int b = 0; b < L.nsub; ++b)
      for (int dz = -kSearch; dz <= kSearch; ++dz)
        for (int dy = -kSearch; dy <= kSearch; ++dy)
          for (int dx = -kSearch; dx <= kSearch; ++dx) {
            const int s = slot(b, dx, dy, dz);
            if (!used[s]) continue;
            Tap t;
            t.b = b;
            t.d[0] = dx;
            t.d[1] = dy;
            t.d[2] = dz;
            bool zero = true;
            for (int k = 0; k < 9; ++k) {
              t.J[k] = acc[(size_t)s * 9 + k];
              zero = zero && t.J[k] == 0.0;
            }
            if (zero) continue;
            c->taps[a].push_back(t);
            c->radius[0] = std::max(c->radius[0], abs(dx));
            c->radius[1] = std::max(c->radius[1], abs(dy));
            c->radius[2] = std::max(c->radius[2], abs(dz));
          }
  }
  c->tables_version = c->ham_version;
}

void free_plan(sx_ctx *c) {
  if (c->stencil) stencil_free(c);
  if (c->fft) fft_free(c);
  if (c->tc) tc_free(c);
  cudaFree(c->d_min);
  c->d_min = nullptr;
  cudaFree(c->d_path);
  c->d_path = nullptr;
  c->path_bytes = 0;
  c->path_vp_nimg = 0;
  cudaFree(c->d_taps);
  cudaFree(c->d_tap_off);
  cudaFree(c->d_work);
  cudaFree(c->d_field);
  cudaFree(c->d_partial);
  cudaFree(c->d_status);
  c->d_status = nullptr;
  cudaFree(c->d_host_S[0]);
  cudaFree(c->d_host_S[1]);
  c->d_taps = nullptr;
  c->d_tap_off = nullptr;
  c->d_work = c->d_field = c->d_partial = nullptr;
  c->d_host_S[0] = c->d_host_S[1] = nullptr;
  c->planned = 0;
}

bool is_iso(const double J[9]) {
  return J[1] == 0.0 && J[2] == 0.0 && J[3] == 0.0 && J[5] == 0.0 && J[6] == 0.0 && J[7] == 0.0 && J[0] == J[4] &&
         J[4] == J[8];
}

int check_ready(const sx_ctx *c) {
  if (!c) return set_error(SX_ERR_ARG, "null context");
  if (!c->planned) return set_error(SX_ERR_STATE, "no plan: call sx_plan first");
  if (c->plan_version != c->ham_version)
    return set_error(SX_ERR_STATE, "Hamiltonian changed since sx_plan: plan again");
  return SX_OK;
}

bool overlaps(const void *p, size_t pbytes, const void *q, size_t qbytes) {
  const char *a = (const char *)p, *b = (const char *)q;
  return a < b + qbytes && b < a + pbytes;
}
bool overlaps(const void *p, const void *q, size_t bytes) { return overlaps(p, bytes, q, bytes); }

int check_spin_ptr(const void *p, const char *name) {
  if (!p) return set_error(SX_ERR_ARG, std::string(name) + " is null");
  if (((uintptr_t)p) & 7u) return set_error(SX_ERR_ARG, std::string(name) + " is not 8-byte aligned");
  return SX_OK;
}

int make_heun_const(const sx_ctx *c, const sx_llg_params *p, HeunConst &h) {
  if (!p) return set_error(SX_ERR_ARG, "null LLG parameters");
  if (!(p->dt_fs > 0.0) || !isfinite(p->dt_fs)) return set_error(SX_ERR_ARG, "dt must be positive");
  if (!(p->alpha >= 0.0) || !isfinite(p->alpha)) return set_error(SX_ERR_ARG, "alpha must be >= 0");
  if (!(p->T_kelvin >= 0.0) || !isfinite(p->T_kelvin)) return set_error(SX_ERR_ARG, "T must be >= 0");
  memset(&h, 0, sizeof(h));
  h.dt = p->dt_fs;
  h.alpha = p->alpha;
  h.g = -kGamma / (1.0 + p->alpha * p->alpha);
  h.seed = p->seed;
  h.replica = p->replica;
  h.thermal = p->T_kelvin > 0.0 && p->alpha > 0.0;
  for (int s = 0; s < c->lat.nsub; ++s)
    h.sigma[s] = h.thermal ? sqrt(2.0 * p->alpha * kKB * p->T_kelvin / (kGamma * c->lat.mu[s] * kMuB * p->dt_fs))
                           : 0.0;
  return SX_OK;
}

cudaError_t backend_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st) {
  if (c->backend == SX_BACKEND_STENCIL) return stencil_field(c, S, b, onsite, st);
  if (c->backend == SX_BACKEND_FFT) return fft_field(c, S, b, onsite, st);
  if (c->backend == SX_BACKEND_IGEMM_TC) return tc_field(c, S, b, onsite, st);
  return gather_field(c, S, b, onsite, st);
}

cudaError_t backend_field_batch(const sx_ctx *c, const double *S, double *b, int count, long long stride,
                                bool onsite, cudaStream_t st) {
  if (c->backend == SX_BACKEND_STENCIL) return stencil_field_batch(c, S, b, count, stride, onsite, st);
  for (int k = 0; k < count; ++k) {
    cudaError_t e = backend_field(c, S + stride * k, b + stride * k, onsite, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t backend_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                         cudaStream_t st) {
  if (c->backend == SX_BACKEND_STENCIL) return stencil_heun_step(c, src, dst, h, step, st);
  if (c->backend == SX_BACKEND_FFT) return fft_heun_step(c, src, dst, h, step, st);
  if (c->backend == SX_BACKEND_IGEMM_TC) return tc_heun_step(c, src, dst, h, step, st);
  return gather_heun_step(c, src, dst, h, step, st);
}

}  // namespace
}  // namespace sx

using namespace sx;

extern "C" {

const char *sx_last_error(void) { return g_err.c_str(); }

int sx_create(sx_ctx **out, const sx_lattice *lat) {
  if (!out || !lat) return set_error(SX_ERR_ARG, "null argument");
  *out = nullptr;
  if (lat->nsub < 1 || lat->nsub > SX_MAX_SUB) return set_error(SX_ERR_ARG, "nsub must be in 1..SX_MAX_SUB");
  for (int k = 0; k < 3; ++k)
    if (lat->n[k] < 1) return set_error(SX_ERR_ARG, "every n[k] must be >= 1");
  if ((int64_t)lat->n[0] * lat->n[1] * lat->n[2] * lat->nsub > ((int64_t)1 << 40))
    return set_error(SX_ERR_ARG, "lattice too large");
  if (!(fabs(cell_volume(*lat)) > 0.0)) return set_error(SX_ERR_ARG, "singular cell");
  for (int s = 0; s < lat->nsub; ++s)
    if (!(lat->mu[s] > 0.0)) return set_error(SX_ERR_ARG, "mu must be positive");
  sx_ctx *c = new (std::nothrow) sx_ctx();
  if (!c) return set_error(SX_ERR_OOM, "host allocation failed");
  c->lat = *lat;
  for (int k = 0; k < 3; ++k) c->lat.pbc[k] = lat->pbc[k] ? 1 : 0;
  double scale = 0.0;
  for (int k = 0; k < 3; ++k) scale = std::max(scale, length(lat->a[k]));
  c->tol = 1e-9 * scale;
  compute_shells(c);
  Geo &g = c->geo;
  g.nx = lat->n[0];
  g.ny = lat->n[1];
  g.nz = lat->n[2];
  g.nsub = lat->nsub;
  g.px = c->lat.pbc[0];
  g.py = c->lat.pbc[1];
  g.pz = c->lat.pbc[2];
  g.ncell = (int64_t)g.nx * g.ny * g.nz;
  g.nsite = g.ncell * g.nsub;
  c->ham_version = 1;
  *out = c;
  return SX_OK;
}

void sx_destroy(sx_ctx *c) {
  if (!c) return;
  if (c->planned) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(c->device);
    free_plan(c);
    cudaSetDevice(cur);
  }
  delete c;
}

int sx_num_shells(const sx_ctx *c) { return c ? c->nshell : set_error(SX_ERR_ARG, "null context"); }

double sx_shell_radius(const sx_ctx *c, int shell) {
  if (!c || shell < 1 || shell > c->nshell) return -1.0;
  return c->shell_r[shell - 1];
}

int sx_add_shell_exchange(sx_ctx *c, int shell, double J) {
  if (!c) return set_error(SX_ERR_ARG, "null context");
  if (shell < 1 || shell > SX_MAX_SHELL || shell > c->nshell) return set_error(SX_ERR_ARG, "shell out of range");
  if (c->shell_r[shell - 1] > search_reach(c->lat)) return set_error(SX_ERR_ARG, "shell beyond the bond search box");
  if (!isfinite(J)) return set_error(SX_ERR_ARG, "J must be finite");
  c->shellJ[shell - 1] += J;
  c->ham_version++;
  return SX_OK;
}

int sx_add_dmi(sx_ctx *c, int shell, int kind, double D) {
  if (!c) return set_error(SX_ERR_ARG, "null context");
  if (shell < 1 || shell > SX_MAX_SHELL || shell > c->nshell) return set_error(SX_ERR_ARG, "shell out of range");
  if (kind != SX_DMI_INTERFACIAL && kind != SX_DMI_BULK) return set_error(SX_ERR_ARG, "unknown DMI kind");
  if (c->dmiD[shell - 1] != 0.0 && c->dmi_kind[shell - 1] != kind)
    return set_error(SX_ERR_ARG, "one DMI kind per shell");
  if (c->shell_r[shell - 1] > search_reach(c->lat)) return set_error(SX_ERR_ARG, "shell beyond the bond search box");
  if (!isfinite(D)) return set_error(SX_ERR_ARG, "D must be finite");
  c->dmi_kind[shell - 1] = kind;
  c->dmiD[shell - 1] += D;
  c->ham_version++;
  return SX_OK;
}

int sx_add_bonds(sx_ctx *c, const sx_bond *bonds, size_t n) {
  if (!c || (n && !bonds)) return set_error(SX_ERR_ARG, "null argument");
  for (size_t i = 0; i < n; ++i) {
    const sx_bond &o = bonds[i];
    if (o.a < 0 || o.b < 0 || o.a >= c->lat.nsub || o.b >= c->lat.nsub)
      return set_error(SX_ERR_ARG, "bond sublattice out of range");
    if (o.a == o.b && o.d[0] == 0 && o.d[1] == 0 && o.d[2] == 0) return set_error(SX_ERR_ARG, "self bond");
    for (int k = 0; k < 3; ++k)
      if (abs(o.d[k]) > kSearch) return set_error(SX_ERR_ARG, "bond offset beyond 4 cells");
    for (int k = 0; k < 9; ++k)
      if (!isfinite(o.J[k])) return set_error(SX_ERR_ARG, "bond tensor must be finite");
  }
  c->bonds.insert(c->bonds.end(), bonds, bonds + n);
  c->ham_version++;
  return SX_OK;
}

int sx_set_zeeman(sx_ctx *c, const double B[3]) {
  if (!c || !B) return set_error(SX_ERR_ARG, "null argument");
  for (int k = 0; k < 3; ++k) {
    if (!isfinite(B[k])) return set_error(SX_ERR_ARG, "B must be finite");
    c->B[k] = B[k];
  }
  c->ham_version++;
  return SX_OK;
}

int sx_set_anisotropy(sx_ctx *c, int sub, double K, const double axis[3]) {
  if (!c || !axis) return set_error(SX_ERR_ARG, "null argument");
  if (sub < 0 || sub >= c->lat.nsub) return set_error(SX_ERR_ARG, "sublattice out of range");
  const double len = length(axis);
  if (!(len > 0.0) || !isfinite(K)) return set_error(SX_ERR_ARG, "bad anisotropy axis or constant");
  c->K[sub] = K;
  for (int k = 0; k < 3; ++k) c->axis[sub][k] = axis[k] / len;
  c->ham_version++;
  return SX_OK;
}

int sx_set_dipolar(sx_ctx *c, int enable) {
  if (!c) return set_error(SX_ERR_ARG, "null context");
  c->dipolar = enable ? 1 : 0;
  c->ham_version++;
  return SX_OK;
}

int sx_get_taps(sx_ctx *c, int a, sx_tap *out, int cap) {
  if (!c) return set_error(SX_ERR_ARG, "null context");
  if (a < 0 || a >= c->lat.nsub) return set_error(SX_ERR_ARG, "sublattice out of range");
  if (cap > 0 && !out) return set_error(SX_ERR_ARG, "null output");
  if (c->tables_version != c->ham_version) build_tables(c);
  const std::vector<Tap> &T = c->taps[a];
  for (int i = 0; i < (int)T.size() && i < cap; ++i) {
    out[i].a = a;
    out[i].b = T[i].b;
    for (int k = 0; k < 3; ++k) out[i].d[k] = T[i].d[k];
    for (int k = 0; k < 9; ++k) out[i].J[k] = T[i].J[k];
  }
  return (int)T.size();
}

int sx_plan(sx_ctx *c, int backend, int prec) {
  if (!c) return set_error(SX_ERR_ARG, "null context");
  if (backend < SX_BACKEND_GATHER || backend > SX_BACKEND_FFT) return set_error(SX_ERR_ARG, "unknown backend");
  if (prec < SX_PREC_FP64 || prec > SX_PREC_BF16) return set_error(SX_ERR_ARG, "unknown precision");
  if ((backend == SX_BACKEND_GATHER || backend == SX_BACKEND_STENCIL) && prec > SX_PREC_FP32)
    return set_error(SX_ERR_UNSUPPORTED, "TF32/BF16 fields need the tensor-core backend");
  if (backend == SX_BACKEND_IGEMM_TC && prec != SX_PREC_BF16 && prec != SX_PREC_TF32)
    return set_error(SX_ERR_UNSUPPORTED, "the tensor-core backend computes the field in BF16 or TF32");
  if (c->dipolar && backend != SX_BACKEND_FFT)
    return set_error(SX_ERR_UNSUPPORTED, "the dipolar term needs the FFT backend");
  if (c->tables_version != c->ham_version) build_tables(c);
  for (int a = 0; a < c->lat.nsub; ++a)
    if ((int)c->taps[a].size() > kMaxTaps) return set_error(SX_ERR_UNSUPPORTED, "too many taps per sublattice");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (c->planned) {
    int cur = dev;
    cudaSetDevice(c->device);
    free_plan(c);
    cudaSetDevice(cur);
  }
  c->device = dev;
  c->backend = backend;
  c->prec = prec;
  const Geo &g = c->geo;

  // on-site constants
  OnSite &os = c->onsite;
  memset(&os, 0, sizeof(os));
  for (int s = 0; s < c->lat.nsub; ++s) {
    const double mm = c->lat.mu[s] * kMuB;
    for (int k = 0; k < 3; ++k) {
      os.zee[s][k] = mm * c->B[k];
      os.axis[s][k] = c->axis[s][k];
    }
    os.twoK[s] = 2.0 * c->K[s];
    os.inv_mm[s] = 1.0 / mm;
  }

  // directed taps for the gather path
  std::vector<DevTap> dt;
  std::vector<int> off(1, 0);
  for (int a = 0; a < c->lat.nsub; ++a) {
    for (const Tap &t : c->taps[a]) {
      DevTap d;
      memset(&d, 0, sizeof(d));
      d.b = t.b;
      d.dx = t.d[0];
      d.dy = t.d[1];
      d.dz = t.d[2];
      d.iso = is_iso(t.J);
      for (int k = 0; k < 9; ++k) {
        d.J[k] = t.J[k];
        d.Jf[k] = (float)t.J[k];
      }
      dt.push_back(d);
    }
    off.push_back((int)dt.size());
  }
  const size_t N3 = 3 * (size_t)g.nsite;
  c->nblock_red = reduce_blocks(g.nsite);
#define SX_TRY(call, what)          \
  do {                              \
    e = (call);                     \
    if (e != cudaSuccess) {         \
      free_plan(c);                 \
      return cuda_error(e, what);   \
    }                               \
  } while (0)
  SX_TRY(cudaMalloc(&c->d_taps, sizeof(DevTap) * std::max<size_t>(1, dt.size())), "cudaMalloc taps");
  SX_TRY(cudaMalloc(&c->d_tap_off, sizeof(int) * off.size()), "cudaMalloc tap offsets");
  if (!dt.empty()) SX_TRY(cudaMemcpy(c->d_taps, dt.data(), sizeof(DevTap) * dt.size(), cudaMemcpyHostToDevice), "copy taps");
  SX_TRY(cudaMemcpy(c->d_tap_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice), "copy offsets");
  if (backend == SX_BACKEND_GATHER) SX_TRY(cudaMalloc(&c->d_work, 2 * N3 * sizeof(double)), "cudaMalloc Heun workspace");
  SX_TRY(cudaMalloc(&c->d_field, N3 * sizeof(double)), "cudaMalloc field workspace");
  SX_TRY(cudaMalloc(&c->d_partial, (3 * c->nblock_red + 8) * sizeof(double)), "cudaMalloc reduction partials");
  SX_TRY(cudaMalloc(&c->d_status, sizeof(int)), "cudaMalloc status word");
  SX_TRY(cudaMemset(c->d_status, 0, sizeof(int)), "clear status word");
  c->launches_per_step = 2;
  if (backend != SX_BACKEND_GATHER) {
    const int rc = backend == SX_BACKEND_STENCIL ? stencil_plan(c) : backend == SX_BACKEND_FFT ? fft_plan(c) : tc_plan(c);
    if (rc != SX_OK) {
      free_plan(c);
      return rc;
    }
  }
#undef SX_TRY
  c->planned = 1;
  c->plan_version = c->ham_version;
  ++c->plan_gen;
  return SX_OK;
}

int sx_set_stencil_scheme(sx_ctx *c, int scheme) {
  if (!c) return set_error(SX_ERR_ARG, "null context");
  if (scheme != SX_STENCIL_AUTO && scheme != SX_STENCIL_FUSED && scheme != SX_STENCIL_TWO_PASS)
    return set_error(SX_ERR_ARG, "unknown stencil scheme");
  if (c->planned && c->backend == SX_BACKEND_STENCIL) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(c->device);
    const int old = c->opt_scheme, old_eff = stencil_scheme(c);
    c->opt_scheme = scheme;
    int rc = stencil_set_scheme(c, scheme);
    if (rc != SX_OK) {
      c->opt_scheme = old;
      stencil_set_scheme(c, old_eff);
    }
    cudaSetDevice(cur);
    return rc;
  }
  c->opt_scheme = scheme;
  return SX_OK;
}

int sx_autotune(sx_ctx *c, const double *S, double *S_scratch, const sx_llg_params *p, int steps, double times_ms[2],
                void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(S, "S")) || (rc = check_spin_ptr(S_scratch, "S_scratch"))) return rc;
  if (overlaps(S, S_scratch, 3 * (size_t)c->geo.nsite * sizeof(double)))
    return set_error(SX_ERR_ARG, "S and S_scratch overlap");
  if (steps < 1) return set_error(SX_ERR_ARG, "steps must be >= 1");
  HeunConst h;
  if ((rc = make_heun_const(c, p, h))) return rc;
  if (times_ms) times_ms[0] = times_ms[1] = -1.0;
  if (c->backend != SX_BACKEND_STENCIL && c->backend != SX_BACKEND_IGEMM_TC) return SX_STENCIL_FUSED;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // mean step time of the current tile shape: one warm-up step, then `steps` timed steps S -> S_scratch
  auto time_steps = [&](double *ms_out) {
    if ((e = backend_step(c, S, S_scratch, h, 0, st)) != cudaSuccess) return;
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = backend_step(c, S, S_scratch, h, (uint64_t)k, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms / steps;
  };
  int result = SX_STENCIL_FUSED;
  if (c->backend == SX_BACKEND_STENCIL) {
    // scheme x z chunk x launch shape (z-chunked grid or balanced schedule over 1 or 2 x the CTA slots)
    const TileChoice keep = stencil_current_tiles(c);
    const int keep_tz = stencil_fused_tz(c);
    TileChoice best = keep;
    double best_ms = -1.0;
    for (const TileChoice &t : stencil_tile_candidates(c, h.thermal != 0)) {
      if (e != cudaSuccess) break;
      if (stencil_apply_tiles(c, t) != SX_OK) continue;  // e.g. no room for the two-pass workspace
      double ms = 0.0;
      time_steps(&ms);
      if (e != cudaSuccess) break;
      double &slot = times_ms ? times_ms[t.scheme - 1] : ms;
      if (times_ms && (slot < 0.0 || ms < slot)) slot = ms;
      if (best_ms < 0.0 || ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    // the best shape with the other plane stagings of the pass kernels (tensor copies or site by site for
    // the predictor and for the corrector), kept only when at least 1% faster
    const TileChoice top = best;
    for (int mask = 0; mask < 4 && e == cudaSuccess && best_ms >= 0.0 && top.scheme == SX_STENCIL_TWO_PASS;
         ++mask) {
      if (mask == top.tma) continue;
      TileChoice t = top;
      t.tma = mask;
      if (stencil_apply_tiles(c, t) != SX_OK) continue;
      double ms = 0.0;
      time_steps(&ms);
      if (e == cudaSuccess && ms < 0.99 * best_ms) {
        best_ms = ms;
        best = t;
        if (times_ms) times_ms[t.scheme - 1] = ms;
      }
    }
    stencil_restore_fused_tz(c, keep_tz);  // the two-pass candidates leave the fused chunk as planned
    const int rc2 = stencil_apply_tiles(c, e == cudaSuccess ? best : keep);
    if (e == cudaSuccess && rc2 != SX_OK) rc = rc2;
    c->opt_scheme = stencil_scheme(c);
    result = stencil_scheme(c);
  } else {
    // ring depth x CTAs per SM of the tensor-core tile kernel
    const TcTiles keep = tc_current_tiles(c);
    TcTiles best = keep;
    double best_ms = -1.0;
    for (const TcTiles &t : tc_tile_candidates(c)) {
      if (e != cudaSuccess) break;
      if (tc_apply_tiles(c, t) != SX_OK) continue;
      double ms = 0.0;
      time_steps(&ms);
      if (e != cudaSuccess) break;
      if (best_ms < 0.0 || ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    tc_apply_tiles(c, e == cudaSuccess ? best : keep);
    if (times_ms) times_ms[0] = best_ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_error(e, "autotune");
  if (rc != SX_OK) return rc;
  return result;
}

int sx_set_tiles(sx_ctx *c, const int64_t in[5]) {
  if (!c || !in) return set_error(SX_ERR_ARG, "null argument");
  int rc = check_ready(c);
  if (rc) return rc;
  if (c->backend == SX_BACKEND_STENCIL) {
    if (in[0] != SX_STENCIL_FUSED && in[0] != SX_STENCIL_TWO_PASS) return set_error(SX_ERR_ARG, "unknown scheme");
    if (in[1] < 1 || in[1] > c->geo.nz) return set_error(SX_ERR_ARG, "z chunk must be in 1 .. n[2]");
    if (in[2] < 0 || in[2] > 5) return set_error(SX_ERR_ARG, "two-pass launch shape must be in 0 .. 5");
    if (in[3] != 0 && in[3] != 1) return set_error(SX_ERR_ARG, "noise regeneration flag must be 0 or 1");
    if (in[0] == SX_STENCIL_FUSED && (in[2] != 0 || in[3] != 0))
      return set_error(SX_ERR_ARG, "the fused scheme has no schedule and no stored normals");
    if (in[4] < 0 || in[4] > 3) return set_error(SX_ERR_ARG, "plane staging mask must be in 0 .. 3");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(c->device);
    rc = stencil_apply_tiles(c, {(int)in[0], (int)in[1], (int)in[2], (int)in[3], (int)in[4]});
    cudaSetDevice(cur);
    if (rc == SX_OK) c->opt_scheme = stencil_scheme(c);
    return rc;
  }
  if (c->backend == SX_BACKEND_IGEMM_TC) {
    if (in[0] != 0 || in[3] != 0 || in[4] != 0) return set_error(SX_ERR_ARG, "the tensor-core plan has one scheme");
    if (in[2] != 1 && in[2] != 2) return set_error(SX_ERR_ARG, "CTAs per SM must be 1 or 2");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(c->device);
    rc = tc_apply_tiles(c, {(int)in[1], (int)in[2]});
    cudaSetDevice(cur);
    return rc;
  }
  return set_error(SX_ERR_UNSUPPORTED, "this backend has no tile shapes to set");
}

int sx_plan_tiles(const sx_ctx *c, int64_t out[8]) {
  if (!c || !out) return set_error(SX_ERR_ARG, "null argument");
  int rc = check_ready(c);
  if (rc) return rc;
  for (int k = 0; k < 8; ++k) out[k] = 0;
  if (c->backend == SX_BACKEND_STENCIL) stencil_tiles_info(c, out);
  if (c->backend == SX_BACKEND_IGEMM_TC) tc_tiles_info(c, out);
  return SX_OK;
}

struct sx_batch {
  sx::StencilBatch *sb;
  std::vector<sx_ctx *> ctxs;
  std::vector<int> plan_gens;
  sx_ctx *img_ctx;
  int img_gen;
  int nimg;
};

namespace {
int batch_create(sx_batch **out, sx_ctx *const *ctxs, int nrep, sx_ctx *img_ctx, int nimg) {
  if (!out) return set_error(SX_ERR_ARG, "null output");
  *out = nullptr;
  if (!ctxs || nrep < 1 || nrep > 65536) return set_error(SX_ERR_ARG, "a batch needs 1 .. 65536 contexts");
  if (img_ctx && (nimg < 1 || nimg > 65536)) return set_error(SX_ERR_ARG, "nimg must be in 1 .. 65536");
  for (int r = 0; r < nrep; ++r) {
    int rc = check_ready(ctxs[r]);
    if (rc) return rc;
    if (ctxs[r]->backend != SX_BACKEND_STENCIL)
      return set_error(SX_ERR_UNSUPPORTED, "batched steps run on STENCIL plans only");
    for (int q = 0; q < r; ++q)
      if (ctxs[q] == ctxs[r]) return set_error(SX_ERR_ARG, "a context appears twice in the batch");
  }
  if (img_ctx) {
    int rc = check_ready(img_ctx);
    if (rc) return rc;
    if (img_ctx->backend != SX_BACKEND_STENCIL)
      return set_error(SX_ERR_UNSUPPORTED, "batched images run on STENCIL plans only");
  }
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ctxs[0]->device);
  for (int r = 0; r < nrep; ++r) {
    if (stencil_scheme(ctxs[r]) != SX_STENCIL_TWO_PASS) {
      const int rc = stencil_set_scheme(ctxs[r], SX_STENCIL_TWO_PASS);
      if (rc != SX_OK || stencil_scheme(ctxs[r]) != SX_STENCIL_TWO_PASS) {
        cudaSetDevice(cur);
        return rc != SX_OK ? rc : set_error(SX_ERR_OOM, "two-pass workspace of a batched context");
      }
    }
  }
  sx::StencilBatch *sb = nullptr;
  const int rc = stencil_batch_create(&sb, ctxs, nrep, img_ctx, img_ctx ? nimg : 0);
  cudaSetDevice(cur);
  if (rc != SX_OK) return rc;
  sx_batch *b = new (std::nothrow) sx_batch();
  if (!b) {
    stencil_batch_free(sb);
    return set_error(SX_ERR_OOM, "host allocation failed");
  }
  b->sb = sb;
  b->ctxs.assign(ctxs, ctxs + nrep);
  for (int r = 0; r < nrep; ++r) b->plan_gens.push_back(ctxs[r]->plan_gen);
  b->img_ctx = img_ctx;
  b->img_gen = img_ctx ? img_ctx->plan_gen : 0;
  b->nimg = img_ctx ? nimg : 0;
  *out = b;
  return SX_OK;
}

int batch_check_plans(const sx_batch *b) {
  for (size_t r = 0; r < b->ctxs.size(); ++r) {
    const sx_ctx *c = b->ctxs[r];
    int rc = check_ready(c);
    if (rc) return rc;
    if (c->plan_gen != b->plan_gens[r] || stencil_scheme(c) != SX_STENCIL_TWO_PASS)
      return set_error(SX_ERR_STATE, "a batched context was re-planned: create the batch again");
  }
  if (b->img_ctx) {
    int rc = check_ready(b->img_ctx);
    if (rc) return rc;
    if (b->img_ctx->plan_gen != b->img_gen)
      return set_error(SX_ERR_STATE, "the image context was re-planned: create the batch again");
  }
  return SX_OK;
}
}  // namespace

int sx_batch_create(sx_batch **out, sx_ctx *const *ctxs, int nrep) { return batch_create(out, ctxs, nrep, nullptr, 0); }

int sx_batch_create_with_images(sx_batch **out, sx_ctx *const *ctxs, int nrep, sx_ctx *img_ctx, int nimg) {
  if (!img_ctx) return set_error(SX_ERR_ARG, "null image context");
  return batch_create(out, ctxs, nrep, img_ctx, nimg);
}

void sx_batch_destroy(sx_batch *b) {
  if (!b) return;
  stencil_batch_free(b->sb);
  delete b;
}

int sx_batch_heun_step(sx_batch *b, const double *const *S_in, double *const *S_out, const sx_llg_params *p,
                       uint64_t step, void *stream) {
  if (!b || !S_in || !S_out) return set_error(SX_ERR_ARG, "null argument");
  int rc = batch_check_plans(b);
  if (rc) return rc;
  const int nrep = (int)b->ctxs.size();
  for (int r = 0; r < nrep; ++r) {
    const sx_ctx *c = b->ctxs[r];
    if ((rc = check_spin_ptr(S_in[r], "S_in")) || (rc = check_spin_ptr(S_out[r], "S_out"))) return rc;
    if (overlaps(S_in[r], S_out[r], 3 * (size_t)c->geo.nsite * sizeof(double)))
      return set_error(SX_ERR_ARG, "S_in and S_out of a replica overlap");
  }
  HeunConst h;
  rc = make_heun_const(b->ctxs[0], p, h);
  if (rc) return rc;
  cudaError_t e = stencil_batch_step(b->sb, S_in, S_out, h, step, (cudaStream_t)stream);
  return e == cudaSuccess ? SX_OK : cuda_error(e, "batched Heun step");
}

int sx_batch_bind(sx_batch *b, double *const *S_a, double *const *S_b, const double *images, double *fields,
                  uint32_t replica0) {
  if (!b || !S_a || !S_b) return set_error(SX_ERR_ARG, "null argument");
  int rc = batch_check_plans(b);
  if (rc) return rc;
  const int nrep = (int)b->ctxs.size();
  for (int r = 0; r < nrep; ++r) {
    const size_t bytes = 3 * (size_t)b->ctxs[r]->geo.nsite * sizeof(double);
    if ((rc = check_spin_ptr(S_a[r], "S_a")) || (rc = check_spin_ptr(S_b[r], "S_b"))) return rc;
    if (overlaps(S_a[r], S_b[r], bytes)) return set_error(SX_ERR_ARG, "S_a and S_b of a replica overlap");
  }
  if (b->nimg > 0) {
    if ((rc = check_spin_ptr(images, "images")) || (rc = check_spin_ptr(fields, "fields"))) return rc;
    const size_t bytes = (size_t)b->nimg * 3 * (size_t)b->img_ctx->geo.nsite * sizeof(double);
    if (overlaps(images, fields, bytes)) return set_error(SX_ERR_ARG, "images and fields overlap");
  }
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->ctxs[0]->device);
  rc = stencil_batch_bind(b->sb, S_a, S_b, images, fields, replica0);
  cudaSetDevice(cur);
  return rc;
}

int sx_batch_run(sx_batch *b, const sx_llg_params *p, uint64_t step0, int nsteps, void *stream) {
  if (!b) return set_error(SX_ERR_ARG, "null batch");
  if (nsteps < 1) return set_error(SX_ERR_ARG, "nsteps must be >= 1");
  int rc = batch_check_plans(b);
  if (rc) return rc;
  if (!stencil_batch_bound(b->sb)) return set_error(SX_ERR_STATE, "sx_batch_bind must precede sx_batch_run");
  HeunConst h;
  if ((rc = make_heun_const(b->ctxs[0], p, h))) return rc;
  const cudaError_t e = stencil_batch_run(b->sb, h, step0, nsteps, (cudaStream_t)stream);
  return e == cudaSuccess ? SX_OK : cuda_error(e, "batched run");
}

int sx_batch_status(sx_batch *b, void *stream) {
  if (!b) return set_error(SX_ERR_ARG, "null batch");
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "batch status");
  if (stencil_batch_check_error(b->sb))
    return set_error(SX_ERR_TIMEOUT, "a grid barrier of sx_batch_run gave up; its results are invalid");
  return take_status(b->ctxs[0], (cudaStream_t)stream);
}

int sx_batch_info(const sx_batch *b, int64_t out[4]) {
  if (!b || !out) return set_error(SX_ERR_ARG, "null argument");
  out[0] = (int64_t)b->ctxs.size();
  out[1] = b->nimg;
  out[2] = stencil_batch_persistent(b->sb);
  out[3] = 0;
  return SX_OK;
}

int sx_device_status(sx_ctx *c, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "device status");
  int timed_out = 0;
  if (c->backend == SX_BACKEND_STENCIL) timed_out |= stencil_check_error(c);
  if (c->backend == SX_BACKEND_IGEMM_TC) timed_out |= tc_check_error(c);
  if (timed_out) return set_error(SX_ERR_TIMEOUT, "a bounded device wait gave up; results of that call are invalid");
  return take_status(c, (cudaStream_t)stream);
}

int sx_field(sx_ctx *c, const double *S, void *b, int out_prec, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (out_prec != SX_PREC_FP64 && out_prec != SX_PREC_FP32)
    return set_error(SX_ERR_ARG, "out_prec must be SX_PREC_FP64 or SX_PREC_FP32");
  if ((rc = check_spin_ptr(S, "S"))) return rc;
  if (!b) return set_error(SX_ERR_ARG, "b is null");
  const size_t n3 = 3 * (size_t)c->geo.nsite;
  if (((uintptr_t)b) & (out_prec == SX_PREC_FP64 ? 7u : 3u)) return set_error(SX_ERR_ARG, "b is misaligned");
  if (overlaps(S, n3 * sizeof(double), b, n3 * (out_prec == SX_PREC_FP64 ? sizeof(double) : sizeof(float))))
    return set_error(SX_ERR_ARG, "S and b overlap");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (out_prec == SX_PREC_FP64) {
    e = backend_field(c, S, static_cast<double *>(b), true, st);
  } else if (c->backend == SX_BACKEND_STENCIL) {
    e = stencil_field_f32(c, S, static_cast<float *>(b), true, st);
  } else if (c->backend == SX_BACKEND_IGEMM_TC) {
    e = tc_field_f32(c, S, static_cast<float *>(b), true, st);
  } else {
    e = backend_field(c, S, c->d_field, true, st);
    if (e == cudaSuccess) e = to_f32(c->d_field, static_cast<float *>(b), (int64_t)n3, st);
  }
  return e == cudaSuccess ? SX_OK : cuda_error(e, "field launch");
}

int sx_llg_heun_step(sx_ctx *c, double *S, double *S_scratch, const sx_llg_params *p, uint64_t step0, int nsteps,
                     void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(S, "S")) || (rc = check_spin_ptr(S_scratch, "S_scratch"))) return rc;
  const size_t bytes = 3 * (size_t)c->geo.nsite * sizeof(double);
  if (overlaps(S, S_scratch, bytes)) return set_error(SX_ERR_ARG, "S and S_scratch overlap");
  if (nsteps < 0) return set_error(SX_ERR_ARG, "nsteps must be >= 0");
  HeunConst h;
  if ((rc = make_heun_const(c, p, h))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double *buf[2] = {S, S_scratch};
  if (nsteps >= 2 && c->backend == SX_BACKEND_STENCIL && stencil_persistent_ok(c)) {
    // small lattices: all steps in one cooperative launch
    cudaError_t e = stencil_heun_steps_persistent(c, S, S_scratch, h, step0, nsteps, st);
    if (e != cudaSuccess) return cuda_error(e, "persistent Heun launch");
  } else {
    for (int k = 0; k < nsteps; ++k) {
      cudaError_t e = backend_step(c, buf[k & 1], buf[(k + 1) & 1], h, step0 + (uint64_t)k, st);
      if (e != cudaSuccess) return cuda_error(e, "Heun step launch");
    }
  }
  if (nsteps & 1) {
    cudaError_t e = cudaMemcpyAsync(S, S_scratch, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "copy back");
  }
  return SX_OK;
}

int sx_llg_heun_step_out(sx_ctx *c, const double *S_in, double *S_out, const sx_llg_params *p, uint64_t step,
                         void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(S_in, "S_in")) || (rc = check_spin_ptr(S_out, "S_out"))) return rc;
  if (overlaps(S_in, S_out, 3 * (size_t)c->geo.nsite * sizeof(double)))
    return set_error(SX_ERR_ARG, "S_in and S_out overlap");
  HeunConst h;
  if ((rc = make_heun_const(c, p, h))) return rc;
  cudaError_t e = backend_step(c, S_in, S_out, h, step, (cudaStream_t)stream);
  return e == cudaSuccess ? SX_OK : cuda_error(e, "Heun step launch");
}

int sx_llg_heun_host(sx_ctx *c, double *S_host, const sx_llg_params *p, uint64_t step0, int nsteps, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!S_host) return set_error(SX_ERR_ARG, "S_host is null");
  if (nsteps < 0) return set_error(SX_ERR_ARG, "nsteps must be >= 0");
  HeunConst h;
  if ((rc = make_heun_const(c, p, h))) return rc;
  const size_t bytes = 3 * (size_t)c->geo.nsite * sizeof(double);
  cudaError_t e;
  for (int k = 0; k < 2; ++k)
    if (!c->d_host_S[k]) {
      e = cudaMalloc(&c->d_host_S[k], bytes);
      if (e != cudaSuccess) return cuda_error(e, "cudaMalloc host-path buffers");
    }
  cudaStream_t st = (cudaStream_t)stream;
  if (c->backend == SX_BACKEND_STENCIL) {
    // two-pass stencil plans pipeline chunked transfers against the passes
    e = stencil_heun_host(c, S_host, c->d_host_S[0], c->d_host_S[1], h, step0, nsteps, st);
    if (e == cudaSuccess) {
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e, "stream synchronize");
      return take_status(c, st);
    }
    if (e != cudaErrorNotSupported) return cuda_error(e, "pipelined host-array step");
  }
  if ((e = cudaMemcpyAsync(c->d_host_S[0], S_host, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_error(e, "host to device copy");
  for (int k = 0; k < nsteps; ++k) {
    e = backend_step(c, c->d_host_S[k & 1], c->d_host_S[(k + 1) & 1], h, step0 + (uint64_t)k, st);
    if (e != cudaSuccess) return cuda_error(e, "Heun step launch");
  }
  if ((e = cudaMemcpyAsync(S_host, c->d_host_S[nsteps & 1], bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_error(e, "device to host copy");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e, "stream synchronize");
  return take_status(c, st);
}

int sx_minimise(sx_ctx *c, double *S, double *S_scratch, const sx_min_params *p, int *iters_out,
                double *torque_out, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(S, "S")) || (rc = check_spin_ptr(S_scratch, "S_scratch"))) return rc;
  if (overlaps(S, S_scratch, 3 * (size_t)c->geo.nsite * sizeof(double)))
    return set_error(SX_ERR_ARG, "S and S_scratch overlap");
  if (!p) return set_error(SX_ERR_ARG, "null minimiser parameters");
  if (p->method != SX_MIN_VP && p->method != SX_MIN_DAMPED_LLG) return set_error(SX_ERR_ARG, "unknown method");
  if (!(p->dt > 0.0) || !(p->tol >= 0.0) || p->max_iter < 0 || p->check_every < 1 || !(p->alpha >= 0.0))
    return set_error(SX_ERR_ARG, "bad minimiser parameters");
  return minimise(c, S, S_scratch, p, iters_out, torque_out, (cudaStream_t)stream, backend_field, backend_step);
}

int sx_path_step(sx_ctx *c, double *images, int nimg, const sx_path_params *p, int *iters_out, double *E_host,
                 double *fmax_host, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(images, "images"))) return rc;
  if (!p) return set_error(SX_ERR_ARG, "null path parameters");
  if (nimg < 3 || nimg > path_max_images())
    return set_error(SX_ERR_ARG, "a chain needs 3 .. " + std::to_string(path_max_images()) + " images");
  if (p->method != SX_PATH_STRING && p->method != SX_PATH_GNEB && p->method != SX_PATH_CI_GNEB)
    return set_error(SX_ERR_ARG, "unknown path method");
  if (!(p->dt > 0.0) || !isfinite(p->dt) || !(p->k_spring >= 0.0) || !isfinite(p->k_spring) || !(p->tol >= 0.0) ||
      p->max_iter < 0 || p->check_every < 1)
    return set_error(SX_ERR_ARG, "bad path parameters");
  if (p->optimizer != SX_PATH_STEEPEST && p->optimizer != SX_PATH_VP)
    return set_error(SX_ERR_ARG, "unknown path optimizer");
  if (p->optimizer == SX_PATH_VP && p->method == SX_PATH_STRING)
    return set_error(SX_ERR_UNSUPPORTED, "velocity projection applies to GNEB and CI-GNEB, not the string method");
  double fmax = -1.0;
  std::vector<double> E(nimg);
  cudaError_t e =
      path_run(c, images, nimg, p, iters_out, E.data(), &fmax, (cudaStream_t)stream, backend_field_batch);
  if (e != cudaSuccess) return cuda_error(e, "path step");
  if (E_host) std::copy(E.begin(), E.end(), E_host);
  if (fmax_host) *fmax_host = fmax;
  bool finite = fmax == -1.0 || std::isfinite(fmax);
  for (double v : E) finite = finite && std::isfinite(v);
  if (!finite) return set_error(SX_ERR_NUMERIC, "a path image holds a non-finite spin (non-finite force or energy)");
  return take_status(c, (cudaStream_t)stream);
}

int sx_geodesic(sx_ctx *c, const double *A, const double *B, double *d_host, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(A, "A")) || (rc = check_spin_ptr(B, "B"))) return rc;
  if (!d_host) return set_error(SX_ERR_ARG, "d_host is null");
  cudaError_t e = geodesic(c, A, B, d_host, (cudaStream_t)stream);
  return e == cudaSuccess ? SX_OK : cuda_error(e, "geodesic");
}

int sx_energy(sx_ctx *c, const double *S, double *E_host, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(S, "S"))) return rc;
  if (!E_host) return set_error(SX_ERR_ARG, "E_host is null");
  cudaStream_t st = (cudaStream_t)stream;
  double *out = c->d_partial + 3 * c->nblock_red;
  cudaError_t e = backend_field(c, S, c->d_field, false, st);
  if (e == cudaSuccess) e = reduce_energy(c, S, c->d_field, c->d_partial, c->nblock_red, out, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(E_host, out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "energy");
  if (!std::isfinite(E_host[0])) return set_error(SX_ERR_NUMERIC, "the energy is not finite: a spin is not finite");
  return SX_OK;
}

int sx_torque_max(sx_ctx *c, const double *S, double *out_host, void *stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if ((rc = check_spin_ptr(S, "S"))) return rc;
  if (!out_host) return set_error(SX_ERR_ARG, "out_host is null");
  cudaStream_t st = (cudaStream_t)stream;
  double *out = c->d_partial + 3 * c->nblock_red;
  cudaError_t e = backend_field(c, S, c->d_field, true, st);
  if (e == cudaSuccess) e = reduce_torque(c, S, c->d_field, c->d_partial, c->nblock_red, out, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "torque");
  if (!std::isfinite(*out_host))
    return set_error(SX_ERR_NUMERIC, "the torque maximum is not finite: a spin or field value is not finite");
  return SX_OK;
}

int sx_thermal_normals(uint64_t seed, uint32_t replica, uint64_t site0, int64_t n, uint64_t step, float *eta_dev,
                       void *stream) {
  if (n < 0 || (n > 0 && !eta_dev)) return set_error(SX_ERR_ARG, "bad output");
  cudaError_t e = thermal_normals(seed, replica, site0, n, step, eta_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SX_OK : cuda_error(e, "normals launch");
}

int sx_plan_info(const sx_ctx *c, int64_t out[8]) {
  if (!c || !out) return set_error(SX_ERR_ARG, "null argument");
  int64_t mt = 0;
  for (const auto &v : c->taps) mt = std::max<int64_t>(mt, (int64_t)v.size());
  out[0] = c->geo.nsite;
  out[1] = mt;
  out[2] = c->radius[0];
  out[3] = c->radius[1];
  out[4] = c->radius[2];
  out[5] = c->planned ? c->backend : -1;
  out[6] = c->planned ? c->prec : -1;
  out[7] = c->planned ? c->launches_per_step : 0;
  return SX_OK;
}

}  // extern "C"
