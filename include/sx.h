/*
 * sx.h -- C ABI of the GB300 (sm_103a) atomistic spin library.
 *
 * The library evaluates the effective field of a translation-invariant spin
 * Hamiltonian on a crystal of n[0] x n[1] x n[2] unit cells with nsub
 * sublattices, and advances the spins with the normalised Heun scheme of the
 * (stochastic) Landau-Lifshitz-Gilbert equation.  It follows the Methods
 * section of arXiv 2605.26016 ("SpinX"):
 *   - "Spin Hamiltonian and effective fields": H = H_bil + H_Z + H_ani + H_dip,
 *     H_bil = -1/2 sum_{i,j} S_i^T J_ij S_j over directed bonds with
 *     J_ji = J_ij^T, J_ij = J I + DMI matrix, reduced field b_i = -dH/dS_i in
 *     meV, physical field B_i = b_i / (mu_i mu_B) in tesla;
 *   - "Backend representations": the bilinear field is the multi-channel
 *     convolution b_a(R) = sum_b sum_delta K_ab(delta) S_b(R + delta) over
 *     sublattice channels; open faces drop the missing neighbours;
 *   - "Atomistic spin dynamics": LLG right-hand side and normalised Heun;
 *   - "Stochastic Landau-Lifshitz-Gilbert simulations": thermal field
 *     sigma eta with sigma = sqrt(2 alpha kB T / (gamma mu mu_B dt)).
 *
 * Units: meV, tesla, fs, nm, kelvin.  Constants (CODATA 2018):
 *   mu_B = 5.7883818060e-2 meV/T, gamma = 1.76085963023e-4 rad/(fs T),
 *   k_B = 8.617333262e-2 meV/K.
 *
 * Spin layout.  A spin field is a caller-owned array of 3*nsite doubles in
 * device memory, nsite = nsub*n[2]*n[1]*n[0]: three component planes
 * [c][sub][z][y][x], x fastest (site index ((sub*nz + z)*ny + y)*nx + x).
 * Fields b use the same layout.  Arrays must be 8-byte aligned and must not
 * overlap unless stated.
 *
 * Ownership.  The caller owns every spin and field buffer.  The library owns
 * its context, coupling tables, plans and workspaces; they are allocated by
 * sx_plan and freed by sx_destroy.
 *
 * Errors.  Every call returns an sx_status (0 = SX_OK, negative on error) and
 * sets a thread-local message read with sx_last_error().  No call aborts,
 * throws across the ABI or traps on the device.  Arguments are checked before
 * any work is queued.  Device calls are asynchronous on the given stream
 * (a cudaStream_t passed as void*; NULL = legacy default stream) unless they
 * return a host value, in which case they synchronise that stream.
 *
 * Thread safety.  Calls on one context must not run concurrently.  Distinct
 * contexts are independent.
 */
#ifndef SX_H
#define SX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SX_MAX_SUB 8
#define SX_MAX_SHELL 16

typedef struct sx_ctx sx_ctx;

typedef enum {
  SX_OK = 0,
  SX_ERR_ARG = -1,         /* bad argument, size or layout */
  SX_ERR_UNSUPPORTED = -2, /* valid request the library or the plan cannot serve */
  SX_ERR_OOM = -3,         /* device or host allocation failed */
  SX_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  SX_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
  SX_ERR_NUMERIC = -6,     /* non-finite or zero-length spin met */
  SX_ERR_STATE = -7        /* call out of order (e.g. no plan yet) */
} sx_status;

typedef enum {
  SX_BACKEND_GATHER = 0,   /* per-site gather over the directed-bond table (any range) */
  SX_BACKEND_STENCIL = 1,  /* shared-memory halo stencil, fused Heun step (sparse convolution) */
  SX_BACKEND_IGEMM_TC = 2, /* tcgen05 implicit GEMM (dense convolution) */
  SX_BACKEND_FFT = 3       /* reciprocal-space kernel (FFT convolution, dipolar) */
} sx_backend;

typedef enum {
  SX_PREC_FP64 = 0, /* field, torque and state update in FP64 */
  SX_PREC_FP32 = 1, /* field and torque in FP32, spin state FP64 ("mixed precision") */
  SX_PREC_TF32 = 2, /* field on tensor cores, TF32 inputs, FP32 accumulate; state FP64 */
  SX_PREC_BF16 = 3  /* field on tensor cores, BF16 inputs, FP32 accumulate; state FP64 */
} sx_precision;

typedef enum { SX_DMI_INTERFACIAL = 0, SX_DMI_BULK = 1 } sx_dmi_kind;

/* How the STENCIL backend runs a Heun step.  Both give bit-identical results
 * (the same FP32 field sums in the same order, the same noise, the same FP64
 * renormalisation).
 *  SX_STENCIL_FUSED:    one launch; the predictor runs on the tile plus a halo
 *                       and keeps S~ in shared memory (48 B of HBM traffic per
 *                       spin-step, more arithmetic per site);
 *  SX_STENCIL_TWO_PASS: a predictor pass writes S~, f0 and (thermal steps)
 *                       the normals as FP32 planes, a corrector pass reads
 *                       them (120 B per spin-step, 144 B with noise; no halo
 *                       recomputation); needs a 36 B per site workspace;
 *  SX_STENCIL_AUTO:     two-pass when its workspace can be allocated. */
typedef enum { SX_STENCIL_AUTO = 0, SX_STENCIL_FUSED = 1, SX_STENCIL_TWO_PASS = 2 } sx_stencil_scheme;

/* Crystal.  Cell vectors a[k] are rows in nm; sub_pos are fractional
 * coordinates; mu[s] is the moment of sublattice s in Bohr magnetons
 * ("Spin Hamiltonian and effective fields": mu_i = mu_i mu_B S_i).
 * pbc[k] = 1 makes axis k periodic, 0 makes it open (free faces). */
typedef struct {
  int n[3];
  int pbc[3];
  double a[3][3];
  int nsub;
  double sub_pos[SX_MAX_SUB][3];
  double mu[SX_MAX_SUB];
} sx_lattice;

/* One unordered bond: pair energy -S_a(R)^T J S_b(R + d) for every cell R,
 * J row-major 3x3 in meV.  It is expanded into the directed bonds
 * (a <- b at +d, J) and (b <- a at -d, J^T) ("Spin Hamiltonian and
 * effective fields", ordered-pair form with J_ji^{ba} = J_ij^{ab}). */
typedef struct {
  int a, b;
  int d[3];
  double J[9];
} sx_bond;

/* A directed tap of the convolution kernel K_ab(delta) for target
 * sublattice a ("Backend representations"): b_a(R) += J S_b(R + d). */
typedef struct {
  int a, b;
  int d[3];
  double J[9];
} sx_tap;

/* Heun/LLG parameters ("Atomistic spin dynamics", "Stochastic LLG"):
 * dt in fs, Gilbert damping alpha, temperature in K (0 = deterministic).
 * Thermal noise eta for site i at step t comes from Philox4x32-10 with
 * counter (i_lo, i_hi, t_lo, replica << 8) and key (seed_lo, seed_hi),
 * mapped to (0,1) by (2*(x>>9)+1)*2^-24 and to normals by Box-Muller; the
 * same eta serves the predictor and the corrector. */
typedef struct {
  double dt_fs;
  double alpha;
  double T_kelvin;
  uint64_t seed;
  uint32_t replica;
} sx_llg_params;

/* Static minimisation on the product of unit spheres ("Static optimization
 * and minimum-energy paths"): tangent force f_i = b_i - (b_i.S_i) S_i,
 * exponential-map retraction R(S, u) = cos|u| S + sin|u| u/|u|.
 *  SX_MIN_VP: velocity projection, per iteration
 *      v <- v + dt/2 (f_prev + f), v <- max(v.f, 0)/(f.f) f (system-wide dot
 *      products), S <- R(S, dt v + dt^2/2 f)   (dt: pseudo time, f in meV);
 *  SX_MIN_DAMPED_LLG: normalised Heun steps of the LLG equation at T = 0,
 *      dt in fs, damping alpha. */
typedef enum { SX_MIN_VP = 0, SX_MIN_DAMPED_LLG = 1 } sx_min_method;

typedef struct {
  int method;       /* sx_min_method */
  double dt;        /* VP pseudo time step, or LLG time step in fs */
  double alpha;     /* damping of SX_MIN_DAMPED_LLG (ignored by VP) */
  double tol;       /* stop when max_i |S_i x b_i| < tol (meV) */
  int max_iter;     /* iteration cap */
  int check_every;  /* iterations between convergence checks, >= 1 */
} sx_min_params;

/* Minimum-energy paths ("Static optimization and minimum-energy paths"):
 * a chain of images Y_0 .. Y_{M-1}, each a whole spin field, with fixed
 * endpoints.  Image distance: the geodesic metric
 * d(Y_n, Y_m) = [sum_i arccos^2(S_i^n . S_i^m)]^(1/2).  With f = b - (b.S) S
 * the tangent force of an image, t+ = P(S_{n+1} - S_n), t- = P(S_n - S_{n-1})
 * (P: projection on the tangent plane of each spin) and tau^ the unit path
 * tangent of image n in image space (t+ when E_{n+1} > E_n > E_{n-1}, t- when
 * E_{n+1} < E_n < E_{n-1}, otherwise the energy-weighted sum with the larger
 * of |E_{n+1} - E_n|, |E_{n-1} - E_n| on the side of the higher neighbour;
 * Henkelman and Jonsson's tangent):
 *  SX_PATH_GNEB:    F = f - (f.tau^) tau^ + k (d(n,n+1) - d(n-1,n)) tau^;
 *  SX_PATH_CI_GNEB: as GNEB, but the highest-energy interior image moves
 *                   with F = f - 2 (f.tau^) tau^;
 *  both then move every interior image by S <- R(S, dt F) (exponential map);
 *  SX_PATH_STRING:  S <- R(S, dt f) for every interior image, then the
 *                   interior images are re-placed at equal geodesic arc
 *                   length along the chain by per-site spherical
 *                   interpolation between the two neighbouring old images. */
typedef enum { SX_PATH_STRING = 0, SX_PATH_GNEB = 1, SX_PATH_CI_GNEB = 2 } sx_path_method;

/* Update rule of the GNEB and CI-GNEB iterations.  SX_PATH_STEEPEST: S <- R(S, dt F).  SX_PATH_VP: velocity
 * projection (the minimisation section lists it among the optimisers; the update of sx_minimise) on the force
 * F of all interior images taken as one vector: v' = v + dt/2 (F_prev + F) (0 on the first iteration from
 * rest), v = max(v'.F, 0)/(F.F) F with the dot products over every interior site, S <- R(S, dt v + dt^2/2 F).
 * The velocity is kept as c and the previous force (another chain in the path workspace). */
typedef enum { SX_PATH_STEEPEST = 0, SX_PATH_VP = 1 } sx_path_optimizer;

typedef struct {
  int method;       /* sx_path_method */
  double dt;        /* step of the retraction, rad per meV of force */
  double k_spring;  /* GNEB spring constant, meV per rad (ignored by the string method) */
  double tol;       /* stop when the largest site force |F| is below tol (meV) at a check */
  int max_iter;     /* iteration cap */
  int check_every;  /* iterations between convergence checks, >= 1 */
  int optimizer;    /* sx_path_optimizer: SX_PATH_STEEPEST or SX_PATH_VP (GNEB and CI-GNEB only) */
  int keep_velocity; /* SX_PATH_VP: 1 = continue from the velocity the previous call on this context left
                        (a VP call on a chain of the same number of images), 0 = start at rest */
} sx_path_params;

/* Create a context for a lattice.  Host-only: makes no CUDA call.
 * SX_ERR_ARG for n[k] < 1, nsub outside 1..SX_MAX_SUB, a singular cell. */
int sx_create(sx_ctx **out, const sx_lattice *lat);

/* Release the context, its plan and its device workspaces (NULL is a no-op). */
void sx_destroy(sx_ctx *ctx);

/* Thread-local text of the last error in this thread. */
const char *sx_last_error(void);

/* Number of distance shells found for the lattice and the radius (nm) of
 * shell k (1-based; shell 1 = nearest neighbours).  Shells are the distinct
 * site-to-site distances sorted ascending, ties within 1e-9 of the cell size
 * ("Hopfion calculation": couplings on the first neighbour shells). */
int sx_num_shells(const sx_ctx *ctx);
double sx_shell_radius(const sx_ctx *ctx, int shell);

/* Isotropic exchange J (meV) on every bond of distance shell `shell`
 * (1-based): J_ij = J I.  Accumulates.  SX_ERR_ARG if the shell is out of
 * range or beyond the bond search box (|delta| <= 4 cells). */
int sx_add_shell_exchange(sx_ctx *ctx, int shell, double J);

/* DMI of strength D (meV) on the bonds of shell `shell`: interfacial
 * D_ij = D (z x r_ij) on bonds in the xy plane, bulk D_ij = D r_ij
 * (r_ij the unit bond vector from i to j).  Enters J_ij as the
 * antisymmetric matrix [[0,Dz,-Dy],[-Dz,0,Dx],[Dy,-Dx,0]]
 * ("Spin Hamiltonian and effective fields"). */
int sx_add_dmi(sx_ctx *ctx, int shell, int kind, double D);

/* General 3x3 tensors (symmetric anisotropic exchange, DMI, ...) as n
 * unordered bonds; see sx_bond.  SX_ERR_ARG for a self bond (a == b, d = 0),
 * a sublattice out of range or |d_k| > 4. */
int sx_add_bonds(sx_ctx *ctx, const sx_bond *bonds, size_t n);

/* Uniform external field B (tesla): H_Z = -sum_i mu_i mu_B B.S_i. */
int sx_set_zeeman(sx_ctx *ctx, const double B[3]);

/* Uniaxial anisotropy on sublattice `sub`: H_ani = -sum K (S_i.n)^2,
 * K in meV, axis normalised by the library.  Replaces the previous value. */
int sx_set_anisotropy(sx_ctx *ctx, int sub, double K, const double axis[3]);

/* Point-dipole interaction between all moments, J_ij^dip =
 * (mu0 mu_B^2/4pi) mu_i mu_j (3 r r - I)/r^3, evaluated in reciprocal space
 * (FFT backend only; periodic axes use the minimum image, a separation of
 * exactly half a period is split into its two images with weight 1/2). */
int sx_set_dipolar(sx_ctx *ctx, int enable);

/* Directed taps (the convolution kernel) of target sublattice a after the
 * Hamiltonian is set: writes up to cap taps, returns their total count or
 * a negative status.  Host-only. */
int sx_get_taps(sx_ctx *ctx, int a, sx_tap *out, int cap);

/* Choose backend and precision, build the device tables and workspaces on
 * the current CUDA device.  Must follow every Hamiltonian change and precede
 * every device call.  SX_ERR_UNSUPPORTED for a combination the library cannot
 * serve (e.g. STENCIL with taps beyond its halo, TF32/BF16 without
 * IGEMM_TC); SX_ERR_ARG if a periodic axis is shorter than 2*range+1. */
int sx_plan(sx_ctx *ctx, int backend, int precision);

/* Choose the STENCIL Heun scheme (sx_stencil_scheme) for this and later
 * plans of the context.  On a planned STENCIL context it takes effect at once
 * (allocating or freeing the two-pass workspace); otherwise it is kept for
 * the next sx_plan.  SX_ERR_ARG for an unknown scheme, SX_ERR_OOM when the
 * two-pass workspace cannot be allocated (the plan is left unchanged). */
int sx_set_stencil_scheme(sx_ctx *ctx, int scheme);

/* Time the candidate tile shapes of the plan on the caller's data and keep
 * the fastest.  STENCIL: the Heun scheme (SX_STENCIL_FUSED, TWO_PASS), the z
 * chunk of a CTA, and for the two-pass scheme the launch shape (a z-chunked
 * grid, a balanced schedule over 1 or 2 times the resident CTA slots, or the
 * overlapped launch with z chunks of about n[2]/4 .. n[2]/16 planes) and, at
 * the fastest shape, the other plane stagings (sx_set_tiles in[4]; kept
 * only when at least 1% faster than the plan's site-by-site staging).
 * IGEMM_TC: the depth of the B-operand ring (2..4) and the CTAs per SM (1 or
 * 2).  Each candidate runs `steps` (>= 1) out-of-place steps S -> S_scratch
 * (S is not modified; S_scratch is overwritten) after one warm-up step.
 * times_ms (may be NULL) receives the best mean step time of
 * SX_STENCIL_FUSED and of SX_STENCIL_TWO_PASS (STENCIL), or the best time in
 * times_ms[0] (IGEMM_TC); -1 when not timed.  sx_plan_tiles reports the
 * choice.  Returns the chosen scheme (> 0; SX_STENCIL_FUSED for plans with
 * one scheme) or a negative status.  Other backends are not timed.
 * Synchronises the stream. */
int sx_autotune(sx_ctx *ctx, const double *S, double *S_scratch, const sx_llg_params *p, int steps,
                double times_ms[2], void *stream);

/* A batch of independent replicas that share one Hamiltonian: planned STENCIL
 * contexts with the same lattice family and identical couplings, on-site
 * terms and moments, but their own lattice sizes and boundaries (e.g. an
 * ensemble of cubes of different edge).  One predictor and one corrector
 * launch advance every replica: the CTAs walk a balanced schedule over all
 * replicas' column-plane units.  sx_batch_create switches the contexts to
 * the two-pass scheme; they must outlive the batch and not be re-planned
 * (SX_ERR_STATE).  SX_ERR_ARG for differing couplings, a repeated context or
 * nrep outside 1..65536; SX_ERR_UNSUPPORTED for non-STENCIL plans. */
typedef struct sx_batch sx_batch;
int sx_batch_create(sx_batch **out, sx_ctx *const *ctxs, int nrep);
void sx_batch_destroy(sx_batch *b);

/* One Heun step at `step` for every replica r of the batch: S_out[r] =
 * Heun(S_in[r]) (host arrays of nrep device pointers; S_in[r] and S_out[r]
 * must not overlap).  Replica r draws its noise with replica index
 * p->replica + r; otherwise bit-identical to sx_llg_heun_step_out on its
 * context. */
int sx_batch_heun_step(sx_batch *b, const double *const *S_in, double *const *S_out, const sx_llg_params *p,
                       uint64_t step, void *stream);

/* Ensembles and minimum-energy-path chains in one launch (ensemble scaling of
 * "GPU performance regimes and scaling"; the images of "Static optimization
 * and minimum-energy paths").  A batch created with images also owns nimg
 * spin fields of img_ctx's lattice (a planned STENCIL context with the
 * replicas' lattice family and couplings; it may be one of the replicas),
 * whose fields sx_batch_run evaluates next to the replicas' steps.  Errors as
 * sx_batch_create; SX_ERR_ARG for nimg outside 1..65536. */
int sx_batch_create_with_images(sx_batch **out, sx_ctx *const *ctxs, int nrep, sx_ctx *img_ctx, int nimg);

/* Bind the device buffers of sx_batch_run (host arrays of nrep device
 * pointers): replica r alternates between S_a[r] and S_b[r] (no overlap) and
 * draws its noise with replica index replica0 + r; image k is images + k *
 * 3 nsite_img (doubles, layout of sx_field) and its field, FP64 with on-site
 * terms, goes to fields + k * 3 nsite_img (images and fields NULL for a
 * batch without images).  Uploads the unit table once; synchronous.  The
 * buffers must outlive every sx_batch_run that uses them. */
int sx_batch_bind(sx_batch *b, double *const *S_a, double *const *S_b, const double *images, double *fields,
                  uint32_t replica0);

/* nsteps >= 1 Heun steps (counters step0 .. step0 + nsteps - 1) of every
 * bound replica, S_a -> S_b -> S_a ... (the result is in S_b[r] for odd
 * nsteps, else in S_a[r]), and the field of every bound image, evaluated in
 * the first step's predictor phase.  One persistent cooperative launch: its
 * CTAs walk a balanced schedule of the column-plane units of all replicas and
 * images, with a grid barrier after each predictor and corrector phase; the
 * barrier waits are bounded and report through sx_batch_status.  When the
 * schedule's CTAs cannot all be resident, the same units run as one launch
 * per phase.  Bit-identical to sx_batch_heun_step steps and sx_field calls.
 * No allocation, no host copy and no synchronisation: a call can be captured
 * in a CUDA graph.  SX_ERR_STATE before sx_batch_bind or after a re-plan. */
int sx_batch_run(sx_batch *b, const sx_llg_params *p, uint64_t step0, int nsteps, void *stream);

/* Synchronise the stream.  SX_ERR_TIMEOUT if a grid barrier of sx_batch_run
 * gave up since the last check (its results are invalid), SX_ERR_NUMERIC if a
 * replica state update met a non-finite or zero-length spin, else SX_OK. */
int sx_batch_status(sx_batch *b, void *stream);

/* out[0] replicas, out[1] images, out[2] 1 when sx_batch_run is one
 * persistent launch (0: one launch per phase), out[3] reserved (0). */
int sx_batch_info(const sx_batch *b, int64_t out[4]);

/* Synchronise the stream and report whether a bounded device wait of this
 * context's kernels gave up since the last check (tensor-core MMA waits, the
 * grid barrier of the persistent multi-step stencil launch): SX_ERR_TIMEOUT
 * then, and the results of the calls since the last check are invalid; the
 * flag is cleared.  No kernel of the library traps or spins without bound:
 * such a wait sets the flag and returns instead. */
int sx_device_status(sx_ctx *ctx, void *stream);

/* Reduced effective field b = -dH/dS (meV, see "Spin Hamiltonian and
 * effective fields") of the spin field S, written to b (device, same layout
 * as S).  out_prec selects the element type of b: SX_PREC_FP64 (3*nsite
 * doubles) or SX_PREC_FP32 (3*nsite floats, for field-only callers; the
 * stencil backend writes it from its FP32 sums directly, the others round
 * their field to FP32).  The values are those of the plan precision either
 * way.  S and b must not overlap.  SX_ERR_ARG for another out_prec. */
int sx_field(sx_ctx *ctx, const double *S, void *b, int out_prec, void *stream);

/* nsteps normalised Heun steps of the LLG equation, steps step0 ..
 * step0+nsteps-1 (the step index is the noise counter).  S (device) holds
 * the input and receives the result; S_scratch (device, same size, no
 * overlap) is a caller-owned ping-pong buffer whose content is overwritten.
 * On a STENCIL two-pass plan of a lattice with fewer tile columns than
 * resident CTAs, nsteps >= 2 run in one cooperative launch with a bounded
 * grid barrier between the passes (bit-identical to separate launches;
 * sx_device_status reports a barrier that gave up).
 * SX_ERR_ARG for dt <= 0, alpha < 0, T < 0 or nsteps < 0. */
int sx_llg_heun_step(sx_ctx *ctx, double *S, double *S_scratch, const sx_llg_params *p, uint64_t step0,
                     int nsteps, void *stream);

/* One normalised Heun step out of place: S_out = Heun(S_in) at step `step`.
 * S_in and S_out are device arrays of 3*nsite doubles that must not overlap;
 * S_in is not modified.  Same rules as sx_llg_heun_step. */
int sx_llg_heun_step_out(sx_ctx *ctx, const double *S_in, double *S_out, const sx_llg_params *p, uint64_t step,
                         void *stream);

/* End-to-end variant on HOST memory: copies S_host to the device, runs
 * nsteps Heun steps in library-owned device buffers and copies the result
 * back into S_host.  Synchronises the stream.  S_host may be pinned or
 * pageable; pinned memory gives full copy bandwidth.  On two-pass STENCIL
 * plans with at least 4 z chunks of max(range, 4) planes the copies go in
 * z chunks on two library streams, pipelined against the passes: the first
 * step's predictor chunks start as their planes (and halo planes) arrive,
 * the last step's corrector chunks go back as soon as they are written,
 * uploads and downloads overlapping.  The results are those of whole copies. */
int sx_llg_heun_host(sx_ctx *ctx, double *S_host, const sx_llg_params *p, uint64_t step0, int nsteps,
                     void *stream);

/* Minimise the energy from S (device, in place) with the plan's field
 * backend; S_scratch (device, same size, no overlap) is overwritten.  Stops
 * after max_iter iterations or when max_i |S_i x b_i| < tol at a check.
 * *iters_out receives the iterations done, *torque_out the last measured
 * torque (meV, -1 if never measured).  The first VP call allocates a
 * 48 B/site workspace kept until sx_destroy.  Synchronises the stream.
 * SX_ERR_ARG for dt <= 0, tol < 0, max_iter < 0, check_every < 1 or an
 * unknown method. */
int sx_minimise(sx_ctx *ctx, double *S, double *S_scratch, const sx_min_params *p, int *iters_out,
                double *torque_out, void *stream);

/* Iterations of a path method (see sx_path_params) on a chain of nimg images
 * (3 .. 4096) stored back to back in `images` (device, image n at
 * images + 3*nsite*n, each in the layout of sx_field), in place; images 0 and
 * nimg-1 are not modified.  The field of every interior image is evaluated
 * with the plan's backend each iteration; FP64 plans do the path arithmetic
 * in FP64, other plans in FP32 with the spins kept and renormalised in FP64.
 * Energies and geodesic sums are reduced in FP64 in a fixed order.  Stops
 * after max_iter iterations or when the largest site force of an iteration
 * is below tol (measured every check_every iterations and on the last).
 * *iters_out: iterations done; E_host (nimg doubles, may be NULL): the image
 * energies (meV) of the final chain; *fmax_host: the largest site force |F|
 * (meV) of the last measured iteration, -1 if none ran.  The first call
 * allocates a workspace of one chain (24 B per site per image) plus partial
 * sums, kept until sx_destroy and grown for a longer chain.  Synchronises
 * the stream.  SX_ERR_ARG for nimg out of range, an unknown method, dt <= 0,
 * k_spring < 0, tol < 0, max_iter < 0 or check_every < 1. */
int sx_path_step(sx_ctx *ctx, double *images, int nimg, const sx_path_params *p, int *iters_out, double *E_host,
                 double *fmax_host, void *stream);

/* Geodesic distance d(A, B) = [sum_i arccos^2(A_i . B_i)]^(1/2) between two
 * spin fields of the context's lattice (device, layout of sx_field), in FP64
 * (per-site angle atan2(|A_i x B_i|, A_i . B_i)).  Synchronises the stream. */
int sx_geodesic(sx_ctx *ctx, const double *A, const double *B, double *d_host, void *stream);

/* Total energy in meV and its parts, E_host[0] = total, [1] = bilinear
 * (-1/2 sum S.b_bil), [2] = Zeeman, [3] = anisotropy, [4] = dipolar, reduced
 * in FP64 in a fixed order (deterministic).  The bilinear field is evaluated
 * in the plan precision.  Synchronises the stream. */
int sx_energy(sx_ctx *ctx, const double *S, double *E_host, void *stream);

/* max_i |S_i x b_i| in meV (the force measure of the minimisation and path
 * methods), written to *out_host.  SX_ERR_NUMERIC when a spin or field value
 * is not finite (the maximum propagates NaN instead of skipping it).
 * Synchronises the stream. */
int sx_torque_max(sx_ctx *ctx, const double *S, double *out_host, void *stream);

/* max_i |S_i x b_i| of caller-provided spins S and fields b (device, layout
 * of sx_field, 3*nsite doubles each, no overlap), written to *out_host.  The
 * paper has no counterpart: this is a variant of sx_torque_max for callers
 * that cannot let the library allocate device memory (an application that
 * reserves the GPU's memory up front in its own arena, or a loop that must
 * not absorb cudaMalloc's implicit synchronisation).  It needs no context,
 * calls no allocating routine, and keeps its partial maxima in a fixed
 * 9.7 KB device array in the library image that every GPU loading the
 * library holds until exit.  Each call looks up that array's address
 * (cudaGetSymbolAddress) in the device and context current at the call.
 * Loading: the CUDA driver loads the library's device code into a context on
 * its first use there (lazy module loading) and reserves device memory for
 * it then; a caller that reserves all remaining device memory for its own
 * arena should make one call of this function (or any library call) on each
 * device first.  All calls share the array, so calls that overlap on the GPU
 * race; calls serialised on one stream do not.  SX_ERR_ARG for null or
 * misaligned pointers, overlap, or nsite outside 1..2^40; SX_ERR_NUMERIC when
 * a spin or field value is not finite (the maximum propagates NaN).
 * Synchronises the stream. */
int sx_torque_max_noalloc(const double *S, const double *b, int64_t nsite, double *out_host, void *stream);

/* The thermal normals the Heun step draws: eta for sites site0 .. site0+n-1
 * at step `step`, written as n x 3 floats to eta_dev (device).  The noise is
 * a pure function of (seed, replica, site, step), see sx_llg_params. */
int sx_thermal_normals(uint64_t seed, uint32_t replica, uint64_t site0, int64_t n, uint64_t step, float *eta_dev,
                       void *stream);

/* Set a tile shape directly (e.g. one that sx_autotune chose earlier, without
 * timing again).  STENCIL: in[0] = scheme (SX_STENCIL_FUSED / TWO_PASS),
 * in[1] = z chunk of a CTA (1 .. n[2]), in[2] = two-pass launch shape (0:
 * z-chunked grid, f = 1..4: balanced schedule over f x the resident CTA
 * slots, 5: one persistent launch whose CTAs take predictor and corrector
 * units of in[1] planes from a dependency-ordered queue, so that the
 * issue-bound predictor and the memory-bound corrector share the SMs; it
 * needs edge tile columns (32 cells), rows and the last z chunk at least as
 * wide as the halo, and one context's steps on one stream at a time), in[3] =
 * 1 when the two-pass corrector regenerates the thermal
 * normals (0 for the fused scheme), in[4] = plane staging of the pass
 * kernels, a mask: bit 0 for the predictor and field passes, bit 1 for the
 * corrector; a set bit makes a tile whose load region lies inside the
 * lattice in x and y stage each plane with one tensor copy (TMA), a clear
 * bit makes every tile copy site by site.  IGEMM_TC: in[0] =
 * 0, in[1] = B-ring depth (2..4), in[2] = CTAs per SM (1 or 2), in[3] =
 * in[4] = 0.  Results do not depend on the shape (every shape runs the same
 * per-site arithmetic).  SX_ERR_ARG for values out of range or a layout that
 * does not fit, SX_ERR_OOM when the two-pass workspace cannot be allocated,
 * SX_ERR_UNSUPPORTED for other backends and for in[4] != 0 on a lattice
 * whose n[0] is not a multiple of 4. */
int sx_set_tiles(sx_ctx *ctx, const int64_t in[5]);

/* Tile shape of the plan (after sx_plan or sx_autotune): out[0] = stencil
 * scheme (0 for other backends), out[1..3] = output tile extent in x, y, z
 * (cells; out[3] = 0 when a balanced schedule assigns z ranges), out[4] = CTAs
 * per launch, out[5] = stencil: two-pass launch shape (see sx_set_tiles in[2]),
 * tensor core: B-operand ring depth, out[6] = 1 when the two-pass corrector
 * regenerates the thermal normals instead of reading the predictor's (the
 * same numbers: a pure function of seed, replica, site and step), out[7] =
 * stencil: the plane staging mask of the pass kernels (see sx_set_tiles).
 * Zeros for the other backends. */
int sx_plan_tiles(const sx_ctx *ctx, int64_t out[8]);

/* Plan facts for callers and tests: out[0] = nsite, out[1] = max taps per
 * sublattice, out[2..4] = halo radius per axis (cells), out[5] = backend,
 * out[6] = precision, out[7] = device kernel launches per Heun step. */
int sx_plan_info(const sx_ctx *ctx, int64_t out[8]);

/* ---------------------------------------------------------------------------
 * Convolutional proposer of path chains.
 *
 * The string and GNEB methods ("Static optimization and minimum-energy
 * paths") start from a chain of images between two endpoint states; the
 * usual first chain is the site-wise geodesic interpolation.  The proposer is
 * a small learned map that turns such an interpolated image into a better
 * first guess of the converged image, trained on paths the path method has
 * converged.  It is not part of the paper's method; the paper's geodesic
 * interpolation stays the fallback (sx_cnn_interpolate).
 *
 * Model, for one sublattice on an n[0] x n[1] x n[2] grid with zero padding
 * outside it: per site the input has 10 channels (interpolated image I,
 * endpoint A, endpoint B, path coordinate s); four 3x3x3 convolutions with
 * bias map 10 -> 16 -> 16 -> 16 -> 3 channels, ReLU after the first three;
 * the proposal is P = N[I + Y] per site (Y the last convolution's output) and
 * the training loss is L = mean over samples and sites of (1 - P . T), T the
 * converged image.  Parameters (sx_cnn_num_params() = 19,491 FP32 values):
 * per layer the weights [out][in][dz][dy][dx] (dz, dy, dx = -1, 0, 1 at index
 * 0, 1, 2) then the biases, layers in order.  Inputs and hidden activations
 * are stored in BF16 (round to nearest even of the FP32 value), weights are
 * rounded to BF16 for the tensor-core convolutions, sums are FP32; the
 * normalisation and the loss are FP64.
 *
 * Image layout: a sample is 3 planes of ncell doubles, [c][z][y][x], x
 * fastest (the layout of sx_field for nsub = 1).  Packed inputs X are BF16
 * bit patterns, [sample][z][y][x][16] (32 bytes per site, 16-byte aligned).
 * All arrays are device memory owned by the caller unless stated.
 * ------------------------------------------------------------------------- */
typedef struct sx_cnn sx_cnn;

typedef struct {
  double lr;     /* step size */
  double beta1;  /* first-moment decay, in [0, 1) */
  double beta2;  /* second-moment decay, in [0, 1) */
  double eps;    /* denominator offset, > 0 */
} sx_adam_params;

/* Number of parameters of the proposer (19,491). */
int64_t sx_cnn_num_params(void);

/* Create a proposer for grids of n[0] x n[1] x n[2] sites and batches of up to
 * max_batch samples.  Allocates the parameters (zero), Adam moments,
 * activations (96 B per site of max_batch samples), activation gradients
 * (128 B per site), a packed-input buffer (32 B per site) and weight-gradient
 * partials (about 110 KB per 16 x 16 x 8 block of sites); synchronises the
 * device.  SX_ERR_ARG for n[k] outside 1..4096 or max_batch outside 1..65535. */
int sx_cnn_create(sx_cnn **out, const int n[3], int max_batch);

/* Release the proposer and its device memory (NULL is a no-op). */
void sx_cnn_destroy(sx_cnn *h);

/* Copy sx_cnn_num_params() parameters from host memory, reset the Adam state
 * and rebuild the tensor-core operands.  Synchronises the device. */
int sx_cnn_set_params(sx_cnn *h, const float *params_host);

/* Copy the parameters to host memory.  Synchronises the device. */
int sx_cnn_get_params(sx_cnn *h, float *params_host);

/* Pack nb samples into X: sample b reads I + b*i_stride, A + b*ab_stride,
 * B + b*ab_stride (each 3*ncell doubles; ab_stride = 0 shares one pair of
 * endpoints) and s[b] (device array of nb doubles).  Strides count doubles;
 * i_stride >= 3*ncell, ab_stride >= 0.  Asynchronous.  SX_ERR_ARG for null or
 * misaligned pointers, nb outside 1..max_batch or bad strides. */
int sx_cnn_pack(sx_cnn *h, const double *I, int64_t i_stride, const double *A, const double *B, int64_t ab_stride,
                const double *s, int nb, uint16_t *X, void *stream);

/* Proposals P (nb x 3 x ncell doubles, may equal I) of nb packed samples X
 * with interpolated images I (nb x 3 x ncell).  Synchronises the stream;
 * SX_ERR_TIMEOUT if a bounded tensor-core wait gave up. */
int sx_cnn_forward(sx_cnn *h, const uint16_t *X, const double *I, int nb, double *P, void *stream);

/* Loss of nb packed samples X with interpolated images I and targets T (each
 * nb x 3 x ncell doubles) and its gradient with respect to every parameter:
 * grad (device, sx_cnn_num_params() floats; NULL keeps it in the proposer for
 * sx_cnn_adam_step) and *loss_host (may be NULL).  Weight gradients are
 * reduced in FP64 in a fixed order (deterministic).  Synchronises the stream. */
int sx_cnn_loss_grad(sx_cnn *h, const uint16_t *X, const double *I, const double *T, int nb, float *grad,
                     double *loss_host, void *stream);

/* One Adam update (Kingma and Ba) of the parameters with gradient grad
 * (device; NULL = the proposer's own, from sx_cnn_loss_grad with grad NULL);
 * rebuilds the tensor-core operands.  Asynchronous. */
int sx_cnn_adam_step(sx_cnn *h, const float *grad, const sx_adam_params *p, void *stream);

/* Geodesic interpolation of a chain (nimg x 3 x ncell doubles, in place):
 * interior image k becomes, site by site, the point at s = k/(nimg-1) of the
 * shorter great-circle arc from image 0 to image nimg-1; parallel pairs blend
 * linearly, antiparallel pairs turn through the part of x-hat (y-hat where
 * |A_x| >= 0.9) orthogonal to A.  Asynchronous.  SX_ERR_ARG for nimg < 3 or
 * nimg - 2 > max_batch. */
int sx_cnn_interpolate(sx_cnn *h, double *chain, int nimg, void *stream);

/* sx_cnn_interpolate, then every interior image replaced by the proposer's
 * output for it (in place).  Synchronises the stream. */
int sx_cnn_propose(sx_cnn *h, double *chain, int nimg, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SX_H */
