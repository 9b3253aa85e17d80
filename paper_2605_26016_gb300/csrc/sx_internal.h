// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sx.h"

namespace sx {

// CODATA 2018 constants in the library's units (meV, T, fs, K).
constexpr double kMuB = 5.7883818060e-2;     // meV / T
constexpr double kGamma = 1.76085963023e-4;  // rad / (fs T)
constexpr double kKB = 8.617333262e-2;       // meV / K
constexpr int kSearch = 4;                   // bond search box: cell offsets -4..4
constexpr int kMaxTaps = 512;                // taps per target sublattice
constexpr int kStatusNumeric = 1;            // status-word bit: a state update met a non-finite or zero-length spin

// One directed tap of K_ab(delta) as stored on the device for the gather path.
struct DevTap {
  int b, dx, dy, dz;
  int iso;  // 1: J = j I (only J[0] used)
  int pad;
  double J[9];
  float Jf[9];
  float pad2;
};

// Lattice geometry as seen by kernels.
struct Geo {
  int nx, ny, nz, nsub;
  int px, py, pz;  // periodic flags
  int pad;
  int64_t ncell, nsite;
};

// On-site terms per sublattice: Zeeman mu mu_B B (meV), uniaxial 2K and axis,
// 1/(mu mu_B) to turn the reduced field into tesla.
struct OnSite {
  double zee[SX_MAX_SUB][3];
  double twoK[SX_MAX_SUB];
  double axis[SX_MAX_SUB][3];
  double inv_mm[SX_MAX_SUB];
};

// Heun step constants shared by every backend.
struct HeunConst {
  double dt;
  double g;                     // -gamma / (1 + alpha^2)
  double alpha;
  double sigma[SX_MAX_SUB];     // thermal field amplitude (T); 0 if deterministic
  uint64_t seed;
  uint32_t replica;
  int thermal;
};

struct Tap {
  int b, d[3];
  double J[9];
};

// On-site and Heun constants in a kernel's arithmetic type R, converted once on
// the host so that no kernel spends FP64 conversions on them per site.
template <typename R>
struct OnSiteT {
  R zee[SX_MAX_SUB][3];
  R twoK[SX_MAX_SUB];
  R axis[SX_MAX_SUB][3];
  R inv_mm[SX_MAX_SUB];
};
template <typename R>
struct HeunT {
  R dt, hdt, g, alpha;
  R sigma[SX_MAX_SUB];
  uint64_t seed;
  uint32_t replica;
  int thermal;
};

template <typename R>
inline OnSiteT<R> onsite_cast(const OnSite &o) {
  OnSiteT<R> r;
  for (int a = 0; a < SX_MAX_SUB; ++a) {
    for (int c = 0; c < 3; ++c) {
      r.zee[a][c] = (R)o.zee[a][c];
      r.axis[a][c] = (R)o.axis[a][c];
    }
    r.twoK[a] = (R)o.twoK[a];
    r.inv_mm[a] = (R)o.inv_mm[a];
  }
  return r;
}

template <typename R>
inline HeunT<R> heun_cast(const HeunConst &h) {
  HeunT<R> r;
  r.dt = (R)h.dt;
  r.hdt = (R)(0.5 * h.dt);
  r.g = (R)h.g;
  r.alpha = (R)h.alpha;
  for (int a = 0; a < SX_MAX_SUB; ++a) r.sigma[a] = (R)h.sigma[a];
  r.seed = h.seed;
  r.replica = h.replica;
  r.thermal = h.thermal;
  return r;
}

// Stencil-backend tables (filled by the host planner, consumed by sx_stencil.cu).
struct StencilPlan;
// FFT-backend buffers and kernel spectrum (sx_fft.cu).
struct FftPlan;
// Tensor-core backend plan (sx_tc.cu).
struct TcPlan;

}  // namespace sx

struct sx_ctx {
  sx_lattice lat;
  sx::Geo geo;
  double shell_r[256];
  int nshell;
  double tol;
  double shellJ[SX_MAX_SHELL];
  int dmi_kind[SX_MAX_SHELL];
  double dmiD[SX_MAX_SHELL];
  std::vector<sx_bond> bonds;
  double B[3];
  double K[SX_MAX_SUB];
  double axis[SX_MAX_SUB][3];
  int dipolar;
  int ham_version;

  // tables built from the Hamiltonian
  std::vector<std::vector<sx::Tap>> taps;  // per target sublattice
  int radius[3];
  int tables_version;

  // plan
  int planned;
  int plan_version;
  int plan_gen;  // incremented by every plan and every workspace change (stale-pointer guard)
  int backend, prec;
  int device;
  sx::OnSite onsite;
  sx::DevTap *d_taps;
  int *d_tap_off;
  double *d_work;        // 2 x 3 nsite doubles: Heun predictor state and f0 (gather path)
  double *d_field;       // 3 nsite doubles: field scratch for energy / torque
  double *d_partial;     // reduction partials
  int *d_status;         // status word set by kernels (kStatusNumeric), read and cleared by the host
  double *d_host_S[2];   // device buffers for the host-memory entry point
  int64_t nblock_red;
  sx::StencilPlan *stencil;
  sx::FftPlan *fft;
  sx::TcPlan *tc;
  double *d_min;  // minimiser workspace (velocity, force, partials), allocated on first use
  int opt_scheme;     // stencil Heun scheme requested for the next plan (sx_stencil_scheme)
  double *d_path;     // path-method workspace (second chain, partial sums), allocated on first use
  size_t path_bytes;  // its size
  int path_vp_nimg;   // chain length whose VP velocity the workspace holds (0: none)
  int launches_per_step;
};

namespace sx {

int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);
// Reads the context's status word after the stream's queued work (synchronises the stream) and clears it:
// SX_ERR_NUMERIC when a state update met a non-finite or zero-length spin since the last check.
int take_status(sx_ctx *c, cudaStream_t st);

// gather path (sx_gather.cu)
cudaError_t gather_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st);
cudaError_t gather_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                             cudaStream_t st);
cudaError_t reduce_energy(const sx_ctx *c, const double *S, const double *bbil, double *partial, int64_t nblock,
                          double *out_dev, cudaStream_t st);
cudaError_t reduce_torque(const sx_ctx *c, const double *S, const double *b, double *partial, int64_t nblock,
                          double *out_dev, cudaStream_t st);
int64_t reduce_blocks(int64_t nsite);
cudaError_t thermal_normals(uint64_t seed, uint32_t replica, uint64_t site0, int64_t n, uint64_t step, float *eta,
                            cudaStream_t st);
// out[i] = in[i] rounded to FP32, i < n
cudaError_t to_f32(const double *in, float *out, int64_t n, cudaStream_t st);

// stencil path (sx_stencil.cu)
int stencil_plan(sx_ctx *c);
void stencil_free(sx_ctx *c);
int stencil_set_scheme(sx_ctx *c, int scheme);  // SX_STENCIL_*, on a planned stencil context
int stencil_scheme(const sx_ctx *c);
// the two-pass scheme's persistent multi-step launch (lattices with fewer tile columns than CTA slots)
bool stencil_persistent_ok(const sx_ctx *c);
// Heun steps on a host array with chunked transfers overlapping the two passes; cudaErrorNotSupported
// when the plan does not take that path
cudaError_t stencil_heun_host(const sx_ctx *c, double *S_host, double *dA, double *dB, const HeunConst &h,
                              uint64_t step0, int nsteps, cudaStream_t st);
cudaError_t stencil_heun_steps_persistent(const sx_ctx *c, double *S0, double *S1, const HeunConst &h,
                                          uint64_t step0, int nsteps, cudaStream_t st);
int stencil_check_error(const sx_ctx *c);
// Tile shapes searched by sx_autotune.  Stencil: scheme, z chunk (tz), and for the two-pass scheme
// either a z-chunked grid (sched = 0) or a balanced schedule over sched x the resident CTA slots.
struct TileChoice {
  int scheme, tz, sched;
  int regen;  // two-pass thermal steps: the corrector regenerates the normals instead of reading them
  int tma;    // pass kernels: interior tiles stage their planes with tensor copies
};
std::vector<TileChoice> stencil_tile_candidates(const sx_ctx *c, bool thermal);
int stencil_apply_tiles(sx_ctx *c, const TileChoice &t);
TileChoice stencil_current_tiles(const sx_ctx *c);
int stencil_fused_tz(const sx_ctx *c);                 // z chunk of the fused step and of single field launches
void stencil_restore_fused_tz(sx_ctx *c, int tz);
// out: scheme, tile x, tile y, z chunk (0: schedule), CTAs per launch, schedule factor (0: grid),
// normals regenerated by the corrector
void stencil_tiles_info(const sx_ctx *c, int64_t out[8]);
// Tensor-core tile layouts searched by sx_autotune: ring depth and CTAs per SM.
struct TcTiles {
  int nbuf, ctas;
};
std::vector<TcTiles> tc_tile_candidates(const sx_ctx *c);
int tc_apply_tiles(sx_ctx *c, const TcTiles &t);
TcTiles tc_current_tiles(const sx_ctx *c);
// out: 0, tile x, tile y, tile z, persistent CTAs, ring depth
void tc_tiles_info(const sx_ctx *c, int64_t out[8]);
// batches of replicas sharing one coupling table (two-pass stencil plans)
struct StencilBatch;
// replicas ctxs[0..nrep) and, when img_ctx is set, nimg images of img_ctx's lattice (field only)
int stencil_batch_create(StencilBatch **out, sx_ctx *const *ctxs, int nrep, const sx_ctx *img_ctx, int nimg);
int stencil_batch_bind(StencilBatch *b, double *const *S_a, double *const *S_b, const double *images,
                       double *fields, uint32_t replica0);
int stencil_batch_bound(const StencilBatch *b);
int stencil_batch_persistent(const StencilBatch *b);
cudaError_t stencil_batch_run(StencilBatch *b, const HeunConst &h, uint64_t step0, int nsteps, cudaStream_t st);
int stencil_batch_check_error(StencilBatch *b);
void stencil_batch_free(StencilBatch *b);
cudaError_t stencil_batch_step(StencilBatch *b, const double *const *S_in, double *const *S_out, const HeunConst &h,
                               uint64_t step, cudaStream_t st);
cudaError_t stencil_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st);
// the field written as FP32 by the field pass itself
cudaError_t stencil_field_f32(const sx_ctx *c, const double *S, float *b, bool onsite, cudaStream_t st);
// fields of `count` spin fields stride doubles apart (S, S + stride, ...) into b, b + stride, ... in one launch
cudaError_t stencil_field_batch(const sx_ctx *c, const double *S, double *b, int count, long long stride,
                                bool onsite, cudaStream_t st);
cudaError_t stencil_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                              cudaStream_t st);

// FFT path (sx_fft.cu)
int fft_plan(sx_ctx *c);
void fft_free(sx_ctx *c);
cudaError_t fft_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st);
cudaError_t fft_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                          cudaStream_t st);

typedef cudaError_t (*FieldFn)(const sx_ctx *, const double *, double *, bool, cudaStream_t);
// fields of count spin fields stride doubles apart, written stride doubles apart
typedef cudaError_t (*FieldBatchFn)(const sx_ctx *, const double *, double *, int, long long, bool, cudaStream_t);

// minimum-energy paths (sx_path.cu)
int path_max_images();
cudaError_t path_run(sx_ctx *c, double *img, int nimg, const sx_path_params *p, int *iters_out, double *E_host,
                     double *fmax_host, cudaStream_t st, FieldBatchFn field);
cudaError_t geodesic(const sx_ctx *c, const double *A, const double *B, double *out_host, cudaStream_t st);

// minimisation (sx_min.cu)
int minimise(sx_ctx *c, double *S, double *S_scratch, const sx_min_params *p, int *iters_out, double *torque_out,
             cudaStream_t st, cudaError_t (*field)(const sx_ctx *, const double *, double *, bool, cudaStream_t),
             cudaError_t (*step)(const sx_ctx *, const double *, double *, const HeunConst &, uint64_t,
                                 cudaStream_t));

// tensor-core path (sx_tc.cu)
int tc_plan(sx_ctx *c);
void tc_free(sx_ctx *c);
cudaError_t tc_field(const sx_ctx *c, const double *S, double *b, bool onsite, cudaStream_t st);
cudaError_t tc_field_f32(const sx_ctx *c, const double *S, float *b, bool onsite, cudaStream_t st);
cudaError_t tc_heun_step(const sx_ctx *c, const double *src, double *dst, const HeunConst &h, uint64_t step,
                         cudaStream_t st);
int tc_check_error(const sx_ctx *c);
// cuTensorMapEncodeTiled (a PFN_cuTensorMapEncodeTiled_v12000) from the driver entry point; null when the
// driver does not provide it
void *tensor_map_encode_fn();

}  // namespace sx
