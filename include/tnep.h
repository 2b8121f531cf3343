/*
 * tnep.h -- C ABI of the GB300 (sm_103a) TNEP tensor library.
 *
 * TNEP (arXiv 2312.05233) predicts the dipole mu (rank 1, Eq. 3) and the
 * polarizability / susceptibility alpha (rank 2, Eq. 4) of a structure from
 * the derivative of a neuroevolution-potential "site value" U_i with respect
 * to the pair vectors r_ij = r_j - r_i (Sec. II.A, the partial force):
 *
 *   mu          = - sum_i sum_{j != i} |r_ij|^2 dU_i/dr_ij                  (Eq. 3)
 *   alpha^{uv}  =   sum_i U_i delta^{uv} - sum_i sum_{j != i} r_ij^u dU_i/dr_ij^v   (Eq. 4)
 *
 * U_i = NN(q_i) is a single-hidden-layer tanh network (Eq. 1) of the NEP
 * descriptor q_i.  The paper defers q_i to the NEP papers; this library uses
 * the published NEP form:
 *   f_c(r)  = (1 + cos(pi r / rc)) / 2 for r < rc,  x = 2 (r/rc - 1)^2 - 1,
 *   f_k(r)  = (T_k(x) + 1) f_c(r) / 2,  k = 0..basis   (Chebyshev T_k),
 *   g_n(r)  = sum_k c^{t_i t_j}_{nk} f_k(r)   (separate c for radial/angular),
 *   radial  q_n  = sum_{r_ij < rc_R} g^R_n(r_ij),              n = 0..n_max_R
 *   angular q_nl = sum_{j,k} g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_ijk), l = 1..l_max
 *   4-body  q_n  = sum_{m1+m2+m3=0} (2 2 2; m1 m2 m3) A_n2m1 A_n2m2 A_n2m3,
 *           A_nlm = sum_{r_ij < rc_A} g^A_n(r_ij) Y_lm(r_ij / r_ij)
 *   U_i     = sum_mu w1_mu tanh(sum_nu W0_mu,nu s_nu - b0_mu) - b1,  s = q * q_scaler.
 *
 * The IR and Raman spectra are cosine transforms of the time-origin averaged
 * autocorrelation of mu(t) (Sec. II.F, Eqs. 5-6) and of gamma = Tr(alpha)/3
 * and beta = alpha - gamma I (Sec. II.G, Eqs. 7-9).
 *
 * Conventions for every entry point:
 *   - Every call returns a tnep_status; nothing throws across the ABI.
 *     tnep_last_error() gives a thread-local message for the last failure.
 *   - Positions are float32 Angstrom, [n][3] row-major.  Boxes are
 *     orthorhombic edge lengths [3]; an edge of 0 marks an open
 *     (non-periodic) axis.  A periodic edge shorter than 2 * rc_R returns
 *     TNEP_ERR_BOX_TOO_SMALL (minimum image must be unique).
 *   - Types are int32 in [0, n_types).
 *   - Input and output pointers may be host or device memory (detected with
 *     cudaPointerGetAttributes).  Inputs are borrowed for the duration of the
 *     call and never retained; outputs are owned by the caller.
 *   - tnep_eval* calls are synchronous: results are in `out` when the call
 *     returns.  `stream` (a cudaStream_t, or NULL for the context's own
 *     stream) is the stream the work is ordered on.
 *   - Tensor outputs are float64.  Rank 1: [3] (x, y, z).  Rank 2: [9]
 *     row-major, element (u, v) = alpha^{uv}.
 *   - Pair selection is exact float32: d = p_j - p_i; on a periodic axis
 *     d = d - L * rint(d * (1/L)); r2 = (dx*dx + dy*dy) + dz*dz with every
 *     operation rounded separately (no fused multiply-add); a pair is kept
 *     iff r2 < rc*rc (rounded to float32).  Strict "<" at the cutoff.
 */
#ifndef TNEP_H
#define TNEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNEP_OK = 0,
  TNEP_ERR_INVALID = 1,            /* bad argument (null pointer, size, type index, layout) */
  TNEP_ERR_OOM = 2,                /* device or pinned host allocation failed */
  TNEP_ERR_BOX_TOO_SMALL = 3,      /* periodic edge < 2 rc_R */
  TNEP_ERR_NEIGHBOR_OVERFLOW = 4,  /* neighbour count above the hard cap (TNEP_OPT_MAX_NEIGHBORS) */
  TNEP_ERR_CUDA = 5,               /* a CUDA runtime call failed; see tnep_last_error() */
  TNEP_ERR_TIMEOUT = 6,            /* a bounded wait expired */
  TNEP_ERR_UNSUPPORTED = 7,        /* hyper-parameters without a compiled kernel variant */
  TNEP_ERR_BUSY = 8,               /* serving: request not admitted (slots or memory) */
  TNEP_ERR_NO_DEVICE = 9           /* no CUDA device or not an sm_103 device */
} tnep_status;

typedef struct tnep_ctx tnep_ctx;  /* opaque, owned by the library */

/* One TNEP model.  All arrays are caller-owned and copied by tnep_create.
 *
 * Flat parameter layout (float32), with D = (n_max_R+1) + (n_max_A+1)*(l_max + use_4body)
 * and H = n_hidden:
 *   for each network (n_types networks if per_type_nn, else one):
 *       W0 [H][D] row-major (hidden unit, descriptor component), b0 [H], w1 [H], b1 [1]
 *   c_R [n_types][n_types][n_max_R+1][basis_R+1]   (centre type, neighbour type, n, k)
 *   c_A [n_types][n_types][n_max_A+1][basis_A+1]
 * Descriptor component order: the radial q_n (n = 0..n_max_R); then for
 * l = 1..l_max the angular q_nl over n = 0..n_max_A; then the 4-body q_n.
 */
typedef struct {
  int rank;           /* 1 = dipole (Eq. 3), 2 = polarizability / susceptibility (Eq. 4) */
  int n_max_R;        /* radial channels n = 0..n_max_R */
  int n_max_A;        /* angular channels n = 0..n_max_A */
  int basis_R;        /* radial Chebyshev basis k = 0..basis_R */
  int basis_A;        /* angular Chebyshev basis k = 0..basis_A */
  int l_max;          /* angular orders l = 1..l_max */
  int use_4body;      /* 1 adds the l = 2 four-body invariant */
  int n_hidden;       /* H, hidden tanh units (1..64) */
  int per_type_nn;    /* 1 = one network per centre type, 0 = one shared network */
  const float* params;
  size_t n_params;
  const float* q_scaler;  /* [D] multiplies q before the network, or NULL = ones */
  int mlp_precision;      /* network products W0 s and W0^T v: 0 = FP32 on the CUDA cores;
                             1 = tensor cores (tcgen05), activations and weights rounded to BF16,
                             FP32 accumulation in tensor memory (relative error ~2^-8);
                             2 = tensor cores, both operands split into high + low BF16 parts,
                             three products hi*hi + hi*lo + lo*hi (error ~2^-17).
                             1 and 2 need descriptor dimension <= 32 and n_hidden <= 32. */
} tnep_model_desc;

/* Creates a context on `device` holding `n_models` models that share the
 * cutoffs {rc_R, rc_A} (Angstrom, rc_A <= rc_R) and therefore one neighbour
 * list per structure.  `type_names` may be NULL.  Supported kernels:
 * (n_max_R, n_max_A, basis_R, basis_A, l_max, use_4body) in
 * {(4,4,8,8,4,1), (3,2,6,5,3,1)}; others return TNEP_ERR_UNSUPPORTED.
 * n_types <= 8.  Returns TNEP_ERR_NO_DEVICE without a usable GPU. */
tnep_status tnep_create(const tnep_model_desc* models, int n_models, int n_types,
                        const char* const* type_names, const float cutoffs[2], int device,
                        tnep_ctx** out);

/* Frees every resource of the context (NULL is a no-op). */
void tnep_destroy(tnep_ctx* ctx);

/* Thread-local message describing the last failed call on this thread. */
const char* tnep_last_error(void);

/* Size of one model's output per structure: 3 (rank 1) or 9 (rank 2); 0 for a bad index. */
int tnep_output_dim(const tnep_ctx* ctx, int model);

/* Evaluates every model of the context on `n_frames` frames of `n_atoms` atoms
 * (a trajectory; Sec. II.H "Workflow").
 *   pos   [n_frames][n_atoms][3]
 *   box   [n_frames][3] orthorhombic edges (0 = open axis) or NULL = all open
 *   types [n_atoms], shared by all frames
 *   out   [n_models][n_frames][C_m] float64, C_m = tnep_output_dim(ctx, m);
 *         model m's block starts at n_frames * sum_{m' < m} C_m'.
 * Frames are processed in chunks (TNEP_OPT_FRAMES_PER_BATCH) with host->device
 * copies of the next chunk overlapped with the current one when `pos` is
 * host memory (pinned memory copies asynchronously). */
tnep_status tnep_eval(tnep_ctx* ctx, int n_frames, int n_atoms, const float* pos,
                      const float* box, const int* types, double* out, void* stream);

/* Evaluates every model on `n_structs` structures of uneven size in one pass
 * (fewer than 2^29 atoms in all).
 *   atom_offsets [n_structs + 1] (host memory), structure s owns atoms
 *                [atom_offsets[s], atom_offsets[s+1]); empty structures allowed
 *   pos [N][3], box [n_structs][3] (0 = open axis) or NULL, types [N]
 *   out [n_models][n_structs][C_m] float64 (layout as tnep_eval)
 *   per_atom  NULL, or [n_models][N][C_m] float32 per-atom contributions in
 *             input order: rank 1: -sum_j |r_ij|^2 dU_i/dr_ij; rank 2:
 *             U_i I - sum_j r_ij (x) dU_i/dr_ij (row-major).  Summing them
 *             over a structure gives its tensor. */
tnep_status tnep_eval_batch(tnep_ctx* ctx, int n_structs, const int* atom_offsets,
                            const float* pos, const float* box, const int* types,
                            double* out, float* per_atom, void* stream);

/* General periodic cells (Sec. II.A): triclinic cells, and cells shorter
 * than twice the cutoff.  U_i depends on the pair vectors to every neighbour
 * within the cutoff, so here a neighbour counts once per image
 * r_j + n H (n integer) within the cutoff -- in a small cell an atom can see
 * another one, or itself, several times.
 *   cell [n_structs][9] float32: rows a, b, c of H (A), row-major; a
 *        structure whose nine entries are all 0 is open; NULL = all open
 *   pos  [N][3] anywhere in space (atoms are wrapped into the cell first)
 *   out  [n_models][n_structs][C_m] float64, as tnep_eval_batch
 * Each periodic structure is expanded on the device into its wrapped atoms
 * plus every image within rc_R / d_a of the cell in fractional coordinates
 * (d_a the lattice-plane spacings), and evaluated as an open structure with
 * the images left out of the sums: the cost grows about as
 * (1 + 2 rc_R / d)^3 for a cell of spacing d.  Host or device buffers
 * (atom_offsets host).  Synchronous.
 * Errors: INVALID (degenerate cell |det H| <= 1e-9, bad sizes or types, more
 * than 2^29 atoms after expansion), NEIGHBOR_OVERFLOW, OOM, CUDA. */
tnep_status tnep_eval_batch_cell(tnep_ctx* ctx, int n_structs, const int* atom_offsets, const float* pos,
                                 const float* cell, const int* types, double* out, void* stream);

/* Builds the neighbour lists of a batch (the cell-list and pair-selection
 * steps of the path) and returns them in input atom order for inspection.
 *   counts_R/counts_A [N]: neighbours within rc_R / rc_A
 *   list_R [N][cap_R], list_A [N][cap_A]: neighbour indices (batch-global, input
 *   order), entries beyond the count (or beyond the cap) are left untouched.
 *   The order inside one atom's list is deterministic but unspecified. */
tnep_status tnep_neighbors(tnep_ctx* ctx, int n_structs, const int* atom_offsets,
                           const float* pos, const float* box, int* counts_R, int* counts_A,
                           int* list_R, int cap_R, int* list_A, int cap_A, void* stream);

/* Population evaluation (the training-time use, Sec. II.D): `n_pop` parameter
 * vectors of model `model` (same hyper-parameters, params [n_pop][n_params])
 * on one batch of structures, with neighbour lists built once.
 *   target [n_structs][C] float64 reference tensors
 *   rmse   [n_pop] float64: sqrt(mean over structures and components of
 *          (prediction - target)^2)
 *   out    NULL or [n_pop][n_structs][C] float64 predictions */
tnep_status tnep_eval_population(tnep_ctx* ctx, int model, int n_pop, const float* params,
                                 int n_structs, const int* atom_offsets, const float* pos,
                                 const float* box, const int* types, const double* target,
                                 double* rmse, double* out, void* stream);

/* Training-style population evaluation with resident structures (Sec. II.D:
 * the evolution strategy evaluates a population on the training set every
 * generation).  tnep_population_create builds the neighbour lists and radial
 * moments of the structures once (they do not depend on the parameters),
 * times the candidate launch shapes of the fused kernel (64 or 128 atoms per
 * CTA; atom-block-major or individual-major CTA order) on these structures
 * and keeps the fastest, and captures one generation -- parameter upload,
 * one fused launch over all n_pop x atoms, FP64 reduction, RMSE, read-back --
 * in a CUDA graph.  `params` [n_pop][n_params] (host) is used for the timing.
 * Arguments otherwise as tnep_eval_population. */
typedef struct tnep_population tnep_population;
tnep_status tnep_population_create(tnep_ctx* ctx, int model, int n_pop, const float* params, int n_structs,
                                   const int* atom_offsets, const float* pos, const float* box,
                                   const int* types, const double* target, tnep_population** out);
/* Replays the captured generation for new parameters [n_pop][n_params] (host):
 * rmse [n_pop], out NULL or [n_pop][n_structs][C] (host).  Synchronous. */
tnep_status tnep_population_eval(tnep_population* pop, const float* params, double* rmse, double* out);
/* info[14]: atoms per CTA, CTA order and form chosen (0 = per-pair angular
 * walk, 1 = factored through the angular moments on the CUDA cores, 2 =
 * factored with tensor-core products), the eight timed candidates of the
 * first two forms (ms per generation: walk with 128/atom-major,
 * 128/individual-major, 64/atom-major, 64/individual-major, then the
 * factored form in the same order; -1 = not applicable), last generation's
 * device time (ms), atoms in the structure set, the timed tensor-core form
 * (ms, -1 = not applicable). */
tnep_status tnep_population_info(const tnep_population* pop, double info[14]);
void tnep_population_destroy(tnep_population* pop);

/* ---- Training loop: separable natural evolution strategy (Sec. II.D) ----
 *
 * The paper trains the parameters z (the flat vector of tnep_model_desc.params,
 * d = n_params entries) with SNES on the loss (Sec. II.D, dipole and
 * polarizability losses)
 *     L(z) = RMSE(z) + lambda1 (1/d) sum |z_i| + lambda2 sqrt((1/d) sum z_i^2),
 * RMSE as in tnep_eval_population.  One generation, population size P:
 *     s_k ~ N(0, I), z_k = mu + sigma * s_k;  rank by L ascending (ties: lower k
 *     first; NaN losses rank last), rank 1 = best;
 *     u_r = max(0, ln(P/2 + 1) - ln r) / sum_j max(0, ln(P/2 + 1) - ln j) - 1/P;
 *     mu    += eta_mu * sigma * sum_k u_{r(k)} s_k;
 *     sigma *= exp(eta_sigma / 2 * sum_k u_{r(k)} (s_k^2 - 1)).
 * The normals come from Philox4x64-10 (Salmon et al. 2011): block b (entries
 * 4b..4b+3) of individual k at generation g uses counter (b, k, g, 0) and key
 * (seed, 0); each 64-bit output x gives u = (floor(x / 2^12) + 1/2) 2^-52, and
 * outputs (x0, x1), (x2, x3) give sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b).
 * mu, sigma, s and the losses are float64; each z_k is rounded to float32 for
 * the evaluation. */
typedef struct {
  int n_pop;                  /* P, 2..1024 */
  double eta_mu;              /* <= 0: 1 */
  double eta_sigma;           /* <= 0: (3 + ln d) / (5 sqrt d) */
  double lambda1, lambda2;    /* regularization weights, >= 0 */
  unsigned long long seed;    /* Philox key word 0 */
} tnep_snes_config;

/* Creates a training run of model `model` of ctx on a resident structure set
 * (arguments as tnep_population_create, host or device buffers); mu0 [d] and
 * sigma0 [d] (host, sigma0 > 0) are the initial search distribution.  The
 * whole generation -- sampling, evaluation of the P individuals, loss,
 * ranking and update -- is captured once in a CUDA graph.  Errors: INVALID
 * (bad config or buffers), OOM, CUDA, NEIGHBOR_OVERFLOW, UNSUPPORTED. */
typedef struct tnep_snes tnep_snes;
tnep_status tnep_snes_create(tnep_ctx* ctx, int model, const tnep_snes_config* cfg, const double* mu0,
                             const double* sigma0, int n_structs, const int* atom_offsets, const float* pos,
                             const float* box, const int* types, const double* target, tnep_snes** out);
/* Runs n_gen generations on the device (one graph replay each).  history NULL
 * or [n_gen][3] (host): loss of the best individual, its RMSE, mean loss of
 * the population, per generation.  Synchronous. */
tnep_status tnep_snes_run(tnep_snes* snes, int n_gen, double* history);
/* Copies the current mu [d] and sigma [d] to host buffers (either may be
 * NULL); *generation (may be NULL) = generations run so far. */
tnep_status tnep_snes_state(const tnep_snes* snes, double* mu, double* sigma, long long* generation);
/* info[4]: generations run, d, population size P, device time of the last
 * tnep_snes_run per generation (ms). */
tnep_status tnep_snes_info(const tnep_snes* snes, double info[4]);
void tnep_snes_destroy(tnep_snes* snes);

/* The two SNES steps alone, on device buffers, asynchronous on `stream`.
 * tnep_snes_normals: s [n_pop][dim] float64 standard normals of `generation`.
 * tnep_snes_update: ranks loss [n_pop] and updates mu [dim], sigma [dim] in
 * place from s [n_pop][dim] (eta_sigma <= 0: the default for dim).
 * n_pop in 2..1024, dim >= 1; INVALID for host pointers or bad sizes. */
tnep_status tnep_snes_normals(unsigned long long seed, long long generation, int n_pop, int dim, double* s,
                              void* stream);
tnep_status tnep_snes_update(int n_pop, int dim, const double* loss, const double* s, double* mu, double* sigma,
                             double eta_mu, double eta_sigma, void* stream);

/* Charged molecules (Sec. III.A): the dipole of a molecule with net charge Q
 * depends on the reference point, so dipole models are trained on the dipole
 * relative to the centre of mass, mu_r; the dipole about the origin is
 *     mu = mu_r + Q r_COM,   r_COM = sum_i m_i r_i / sum_i m_i.
 * tnep_set_masses stores one mass per type (any unit; only ratios matter).
 * tnep_add_com_dipole adds Q_s r_COM,s to mu[s * mu_stride + 0..2] in place for
 * each structure s of a batch (for the output of tnep_eval_batch, whose
 * layout is [n_models][n_structs][C_m], pass the rank-1 model's block and
 * mu_stride = 3).
 *   charge [n_structs] float64 in e (0 = neutral, left unchanged); a charged
 *   structure must be open (box row 0 0 0, checked for host buffers).
 *   atom_offsets host; pos, box (may be NULL = all open), types, charge, mu
 *   host or device.  Sums in float64, fixed order.  Synchronous.
 * Errors: INVALID (no masses set, bad sizes, charged periodic structure). */
tnep_status tnep_set_masses(tnep_ctx* ctx, const double* masses);
tnep_status tnep_add_com_dipole(tnep_ctx* ctx, int n_structs, const int* atom_offsets, const float* pos,
                                const float* box, const int* types, const double* charge, double* mu,
                                int mu_stride, void* stream);

/* Spectrum kinds for tnep_spectrum. */
enum {
  TNEP_SPECTRUM_IR = 0,          /* series [T][3] = mu(t); omega^2 * lineshape (Eq. 6) */
  TNEP_SPECTRUM_RAMAN_ISO = 1,   /* series [T][9] = alpha(t); gamma = Tr(alpha)/3 (Eq. 9) */
  TNEP_SPECTRUM_RAMAN_ANISO = 2  /* series [T][9]; Tr[beta(0) beta(t)], beta = alpha - gamma I */
};

/* Autocorrelation + one-sided cosine transform (Sec. II.F-G), float64:
 *   C(tau) = 1/(T - tau) sum_{t=0}^{T-1-tau} x(t).x(t+tau)  (IR: one third of the trace)
 *   S(nu_k) = dt [C(0) + 2 sum_{tau=1}^{M} C(tau) cos(pi k tau / M)],  nu_k = k / (2 M dt)
 * with M = max_lag (0 < M < T; M <= 0 selects T/2), the series mean removed
 * first when subtract_mean != 0.
 *   series   [T][C] (host or device), C = 3 (IR) or 9 (Raman)
 *   freq_cm1 [M+1] frequencies in cm^-1, spec [M+1] (host or device)
 *   acf_out  NULL or [M+1] the autocorrelation itself
 * Once channels x T x (M+1) exceeds 1e9 (channels: IR 3, iso 1, aniso 9) the
 * autocorrelation is taken through a float64 FFT of the zero-padded series
 * (length a power of two >= T + M); it equals the direct sums to rounding. */
tnep_status tnep_spectrum(const double* series, int T, int C, double dt_fs, int kind,
                          int max_lag, int subtract_mean, double* freq_cm1, double* spec,
                          double* acf_out, void* stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of evaluation requests (one structure each): the
 * evaluation of Eqs. 3-4 for many independent structures (Sec. III.C notes
 * that small systems leave a GPU limited by input/output; batching requests
 * that arrive close together is the remedy).  Requests
 * are copied in by tnep_submit and admitted while `max_slots` requests are
 * not exceeded and the estimated device memory of the admitted, unfinished
 * requests stays within `mem_budget_bytes` (else TNEP_ERR_BUSY; retry later).
 * A worker thread keeps up to `n_pipelines` batches in flight, each on its
 * own stream and resident workspace; a free pipeline takes every pending
 * request (up to `max_batch_atoms` atoms) as one batch, so requests that
 * arrive while others run are batched and overlap them on the device.  A
 * structure's result is bitwise the same alone and in any batch.  While a
 * server runs, the context must not be used by other calls.  Results are
 * [n_models][C_m] float64 per request (models in context order). */
typedef struct tnep_server tnep_server;
typedef struct {
  int n_atoms;
  const float* pos;   /* [n_atoms][3] host memory */
  const float* box;   /* [3] orthorhombic edges (0 = open axis) or NULL = open */
  const int* types;   /* [n_atoms] host memory */
} tnep_request;

tnep_status tnep_server_start(tnep_ctx* ctx, size_t mem_budget_bytes, int max_slots, int n_pipelines,
                              int max_batch_atoms, tnep_server** out);
/* Copies the request; TNEP_ERR_BUSY when it cannot be admitted now. */
tnep_status tnep_submit(tnep_server* server, const tnep_request* req, uint64_t* ticket);
/* Non-blocking: *done = 1 and the result in `out` once finished (the ticket is then released);
 * latency_s (may be NULL) = submission to completion, in seconds. */
tnep_status tnep_poll(tnep_server* server, uint64_t ticket, double* out, int* done, double* latency_s);
/* Blocks up to timeout_s seconds; TNEP_ERR_TIMEOUT if the request is not finished by then. */
tnep_status tnep_wait(tnep_server* server, uint64_t ticket, double* out, double timeout_s, double* latency_s);
/* stats[6]: completed requests, batches launched, atoms evaluated, admitted bytes in use,
 * requests in flight, requests pending. */
tnep_status tnep_server_stats(tnep_server* server, double stats[6]);
/* Finishes admitted requests (bounded by their device work), then frees the server.
 * Calls on the server already in progress when the stop begins complete first
 * (a submit is then either served or refused with TNEP_ERR_INVALID); no call
 * may start on the server once tnep_server_stop has been called. */
void tnep_server_stop(tnep_server* server);

/* Polarized Raman (Sec. II.G).  The Stokes cross-section for observed
 * polarization n and incoming polarization eps is
 *     sum_{gamma delta mu nu} n_gamma eps_delta n_mu eps_nu L_{gamma delta mu nu}(omega)   (Eq. 7)
 * with L the Fourier transform of <alpha_{gamma delta}(0) alpha_{mu nu}(t)> (Eq. 8).
 * tnep_raman_tensor computes, for p = (gamma, delta), q = (mu, nu) (row-major
 * index 3 gamma + delta) and tau = 0..M,
 *     C_pq(tau) = 1/(T - tau) sum_{t=0}^{T-1-tau} a_p(t) a_q(t + tau)
 * (each component's mean removed first when subtract_mean != 0) and keeps the
 * part every polarization contraction sees, S_pq = (C_pq + C_qp) / 2, with the
 * cosine transform of tnep_spectrum:
 *     L_pq(nu_k) = dt [S_pq(0) + 2 sum_{tau=1}^{M} S_pq(tau) cos(pi k tau / M)],
 * nu_k = k / (2 M dt), M = max_lag (<= 0: T/2), 0 < M < T.
 *   series   [T][9] float64 alpha(t) or chi(t), row-major 3x3 (host or device)
 *   freq_cm1 [M+1], L [M+1][9][9] (host or device).  Synchronous.
 * Cost: 81 T (M+1) float64 multiply-adds (direct time-origin sums). */
tnep_status tnep_raman_tensor(const double* series, int T, double dt_fs, int max_lag, int subtract_mean,
                              double* freq_cm1, double* L, void* stream);
/* Eq. 7 for n_orient pairs of polarization vectors: n, eps [n_orient][3]
 * (any length; the contraction is quadratic in each), L [max_lag+1][9][9]
 * from tnep_raman_tensor, spec [n_orient][max_lag+1].  Host or device
 * buffers.  Synchronous. */
tnep_status tnep_raman_polarized(const double* L, int max_lag, int n_orient, const double* n, const double* eps,
                                 double* spec, void* stream);
/* Orientation map in Porto notation (Sec. IV, BaZrO3): for a crystal turned
 * by theta (radians) about crystal axis `axis` (0, 1, 2 = x, y, z; the laser
 * direction), with X, Y the next two axes in cyclic order, the incoming
 * polarization is R^T X = cos(theta) X - sin(theta) Y and the observed one is
 * R^T X for Z(XX)Z-bar (spec_parallel) or R^T Y = sin(theta) X + cos(theta) Y
 * for Z(XY)Z-bar (spec_crossed); both [n_theta][max_lag+1].  Host or device
 * buffers.  Synchronous. */
tnep_status tnep_raman_porto_map(const double* L, int max_lag, int n_theta, const double* theta, int axis,
                                 double* spec_parallel, double* spec_crossed, void* stream);

/* Longest series tnep_spectrum_noalloc accepts (its scratch is sized for it). */
#define TNEP_NOALLOC_MAX_T 32768

/* The spectrum tail of tnep_spectrum without any device allocation.  The
 * paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc, such as an MD engine that reserves all device memory for its
 * own arena at start-up, or that computes spectra inside its time-step loop
 * where cudaMalloc / cudaFree would add a device-wide synchronisation.
 *   series [T][C] and the outputs freq_cm1 [M+1], spec [M+1], acf_out [M+1]
 *   (or NULL) must be device memory; arguments and results are as in
 *   tnep_spectrum.  T <= TNEP_NOALLOC_MAX_T, else TNEP_ERR_INVALID.
 * Scratch lives in one file-scope device array of about 3 MB
 * ((12 * TNEP_NOALLOC_MAX_T) doubles) that every GPU which loads the library
 * holds until the process exits.  The first call on a device looks up that
 * device's address of the array (once per device); make that first call
 * before any stream capture.  The call is asynchronous on `stream`: results
 * are ready once the stream has synchronised.  All calls share the one
 * array, so calls that overlap on the GPU (different streams, or different
 * host threads) race on it; order them on one stream.  Nothing from the
 * previous call has to be cleared: every scratch element is written before
 * it is read.  Calls no cudaMalloc, cudaFree or allocating library routine. */
tnep_status tnep_spectrum_noalloc(const double* series, int T, int C, double dt_fs, int kind,
                                  int max_lag, int subtract_mean, double* freq_cm1, double* spec,
                                  double* acf_out, void* stream);

/* Tunables (tnep_set_option / tnep_get_option). */
enum {
  TNEP_OPT_FRAMES_PER_BATCH = 0,    /* frames per device pass in tnep_eval (0 = automatic) */
  TNEP_OPT_MAX_NEIGHBORS = 1,       /* hard cap on neighbours per atom (default 1024); lists grow up to it */
  TNEP_OPT_BLOCK_ATOMS = 2,         /* atoms per CTA of the fused kernel: 64 or 128 (default 128); models whose
                                       network runs on the tensor cores always take 128 (one per product row) */
  TNEP_OPT_LAST_KERNEL_MS = 3,      /* read-only: device time of the tensor kernels (radial moments + fused) of the last call (ms) */
  TNEP_OPT_CELL_DIV = 4,            /* cells of edge rc_R / k with a +-k stencil, k in {1, 2, 3}; stencil cells
                                       farther than the cutoff are skipped (default 1) */
  TNEP_OPT_LAST_KERNEL_LAUNCHES = 5,/* read-only: fused-kernel launches in the last call */
  TNEP_OPT_LAST_NBR_MS = 6,         /* read-only: device time of the cell/neighbour pipeline in the last call (ms) */
  TNEP_OPT_KERNEL_LAUNCHES_TOTAL = 7,/* read-only: kernels launched by this library in this process */
  TNEP_OPT_SKIN = 8,                /* Verlet skin (A) for tnep_eval, default 0.  With a skin s > 0 each pass of
                                       frames builds lists with cutoffs + s for its first frame and re-tests those
                                       candidates under each frame's positions with the exact float32 pair rule,
                                       so every frame still sees exactly the pairs within the cutoffs; if an atom
                                       moved more than s / 2 within a pass, or the box changed, the call redoes
                                       every pass with lists built per frame.  Results agree with s = 0 to float32
                                       rounding (pair order may differ). */
  TNEP_OPT_LAST_SKIN_USED = 9,      /* read-only: 1 if the last tnep_eval used skin lists in every pass */
  TNEP_OPT_POPULATION_FORM = 10,    /* angular form of populations created afterwards: 0 = the fastest by
                                       timing (default), 1 = per-pair walk, 2 = factored through the angular
                                       moments on the CUDA cores, 3 = factored with the angular sums and the
                                       angular share of Eqs. 3-4 as tensor-core products over the individuals
                                       (2 and 3: FP32 network only; 3: standard descriptor sizes and at most 3
                                       types; otherwise the fastest available) */
  TNEP_OPT_CELL_XDIV = 11,          /* k_x in {1, 2, 3, 4} (default 2), used with cell_div = 1: cells of edge
                                       rc_R / k_x along x; for k_x > 1 each atom scans, in each (y, z) row of its
                                       stencil, only the x-cells that meet [x_i - h, x_i + h], h^2 = rc_R^2 -
                                       (distance from atom i to the row)^2.  Same pair sets; list order may differ. */
  TNEP_OPT_ALLOC_COUNT = 12,        /* read-only: device and pinned-host allocations made by the library in this
                                       process so far.  Host-side fault injection: with the environment variable
                                       TNEP_FAULT=oom@N set before the library is loaded, allocation number N
                                       fails once (nothing is allocated, the device is untouched) and the call
                                       making it returns TNEP_ERR_OOM; the context stays usable. */
  TNEP_OPT_WAIT_TRIES = 13,         /* try_wait limit of the device-side waits for the tensor-core network's
                                       products (default 4194304).  A CTA whose wait runs out stores nothing,
                                       waits (with the default limit) for its product to finish, frees its tensor
                                       memory and makes the call return TNEP_ERR_TIMEOUT; 0 makes every such
                                       wait give up at once (used to test that path).  The context stays usable. */
  TNEP_OPT_PAIR_CACHE = 14          /* 1 (default): the fused kernel's forward walk over the angular list stores
                                       each pair's r_ij, 1/|r_ij|, g_n and g_n' (64 bytes for the standard sizes)
                                       in a device buffer of cap_A x 64 bytes per atom that its backward walk
                                       reads back; 0: the backward walk recomputes them.  Results are the same
                                       either way (bit for bit); skipped where the buffer would exceed 16 GB. */
};
tnep_status tnep_set_option(tnep_ctx* ctx, int option, double value);
tnep_status tnep_get_option(const tnep_ctx* ctx, int option, double* value);

#ifdef __cplusplus
}
#endif

#endif /* TNEP_H */
