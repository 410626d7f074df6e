/*
 * compton.h -- C ABI of the GB300 Compton pair-scatter library (libcompton.so).
 *
 * The library implements the data-parallel hot path of the Monte-Carlo
 * Compton-scattering step of a particle-in-cell code (arXiv 2206.02937,
 * Sec. 3.1 and Sec. 3.2): electron and photon macro-particles are binned by
 * collision cell and paired at random inside each cell, every pair gets its
 * probability of interaction from the Klein-Nishina cross section evaluated in
 * the electron rest frame, a Bernoulli trial decides the collision, and the
 * momenta of accepted pairs are updated.  A small fully connected network can
 * replace the probability evaluation (Sec. 2, Sec. 3.2).
 *
 * Units (Sec. 3.2): momenta in m_e c (electron u, photon k; photon energy
 * eps = |k| in m_e c^2), cross sections in units of sigma_T, densities in
 * 1/(sigma_T c t_unit), so that n * sigma * c * dt is dimensionless.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a compton_status; nothing aborts or exits.
 *   - Pointers named *_dev are device pointers owned by the caller; the
 *     library never frees them.  Host pointers are named *_host.
 *   - Calls are asynchronous on the stream they are given (NULL = legacy
 *     default stream) unless stated otherwise.  One context per host thread,
 *     except compton_submit / compton_poll, which are thread-safe.
 *   - Errors found by a kernel (a cell index out of range, ...) are recorded
 *     in a device word of the context; compton_check() synchronises the stream
 *     and reports them.
 *   - All library-owned device memory is allocated in compton_init, within
 *     compton_config.mem_budget_bytes, except the serving pool, allocated
 *     once by compton_serve_start; no other entry point allocates.
 */
#ifndef COMPTON_H
#define COMPTON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared here so this header needs no CUDA. */
typedef struct CUstream_st* compton_stream_t;

typedef enum compton_status {
    COMPTON_OK = 0,
    COMPTON_EINVAL = 1,    /* bad argument (null pointer, size, mode, ...)          */
    COMPTON_ENOMEM = 2,    /* device allocation failed or exceeds the budget        */
    COMPTON_EBUSY = 3,     /* serving: no slot or budget free now; retry later      */
    COMPTON_ETIMEOUT = 4,  /* a bounded device wait gave up                         */
    COMPTON_ERANGE = 5,    /* input out of range (cell index, size beyond capacity) */
    COMPTON_ENOTREADY = 6, /* serving: the request has not finished                 */
    COMPTON_ECUDA = 7,     /* a CUDA call failed; compton_last_error() has the text */
    COMPTON_ENOMODEL = 8   /* surrogate mode requested but no network is loaded     */
} compton_status;

typedef enum compton_mode {
    COMPTON_MODE_PLAIN = 0,    /* analytic probability (Klein-Nishina)      */
    COMPTON_MODE_MLP_FP32 = 1, /* surrogate network, FP32 operands          */
    COMPTON_MODE_MLP_BF16 = 2, /* surrogate network, BF16 operands          */
    COMPTON_MODE_MLP_FP8 = 3,  /* surrogate network, FP8 E4M3 operands      */
    COMPTON_MODE_PNET = 4      /* the paper's 9-12-9 network, FP32          */
} compton_mode;

/* Inputs of the surrogate network (compton_mlp_set_features). */
typedef enum compton_features {
    COMPTON_FEATURES_MOMENTA = 0,   /* the particles' momenta (Sec. 3.2), sgnlog-scaled */
    COMPTON_FEATURES_INVARIANTS = 1 /* ln(x)/8, ln(v)/8 of the pair, zeros elsewhere    */
} compton_features;

typedef struct compton_config {
    int64_t n_cells;             /* number of collision cells C (> 0)                          */
    int64_t max_particles;       /* capacity per species (sizes the sort scratch)              */
    double w_over_v;             /* macro-particle weight / cell volume: the density one
                                    macro-particle adds to its cell                            */
    double dt;                   /* time step                                                  */
    uint64_t seed;               /* Philox key of the whole run                                */
    int32_t device;              /* CUDA device ordinal                                        */
    float gamma_fp64_threshold;  /* electrons with gamma above this get the pair invariants
                                    recomputed in FP64 (0 = always, inf = never)               */
    float collide_fp64_threshold; /* collisions with gamma * eps above this run the boost and
                                    momentum update in FP64, below it in FP32 (whose error
                                    relative to gamma + eps stays below 2e-6 up to 8);
                                    0 = always FP64                                            */
    uint64_t mem_budget_bytes;   /* cap on library-owned device memory (0 = no cap)            */
    int64_t max_train_batch;     /* largest minibatch of compton_mlp_train_step (sizes its
                                    scratch: 2060 bytes per sample); 0 = no training           */
} compton_config;

/* One species in structure-of-arrays form (all device pointers, length n).
 * For photons u* hold the momentum k.  id is a per-particle identifier,
 * unique within the species; it orders particles whose random keys tie.
 * w_dev, optional, holds each macro-particle's weight over the cell volume
 * (the density it adds to its cell; > 0 and finite); NULL gives every
 * particle the context's w_over_v.  With weights the binning carries them
 * along and the scatter step pairs unequal weights (compton_scatter_step). */
typedef struct compton_species {
    float* ux_dev;
    float* uy_dev;
    float* uz_dev;
    int32_t* cell_dev;  /* collision cell in [0, n_cells) */
    uint32_t* id_dev;
    int64_t n;
    float* w_dev;       /* per-particle weight over cell volume, or NULL */
} compton_species;

/* Pair list of one step, produced by compton_bin_pairs.  Its pointers refer to
 * context memory and stay valid until the next compton_bin_pairs on the same
 * context.  Pairs of cell c are the ranks 0..M_c-1 of both species in that
 * cell, M_c = min(N_e,c, N_g,c); pair p has counter id p. */
typedef struct compton_pairs {
    const int32_t* off_e_dev;     /* [n_cells+1] first sorted electron of each cell */
    const int32_t* off_g_dev;     /* [n_cells+1] first sorted photon of each cell   */
    const void* cell_info_dev;    /* [n_cells] per-cell pair offset, starts, density */
    const int32_t* tile_cell_dev; /* per tile of pairs: the cell of its first pair  */
    const int64_t* n_pairs_dev;   /* total pair count (device scalar)               */
    int64_t max_pairs;            /* host-side bound: min(n_e, n_g)                  */
    int64_t n_cells;
} compton_pairs;

/* Counters accumulated by the kernels since the last reset. */
typedef struct compton_stats {
    uint64_t pairs_tested;   /* pairs whose probability was evaluated           */
    uint64_t scatters;       /* pairs that collided                             */
    uint64_t mlp_fallbacks;  /* surrogate pairs outside its range (analytic P)  */
    uint64_t error_flags;    /* bit 0: cell out of range; bit 1: capacity       */
} compton_stats;

/* ---------------------------------------------------------------------- */
/* Context                                                                 */
/* ---------------------------------------------------------------------- */

/* Create a context on cfg->device: allocates the scratch for binning and
 * scattering (about 164 bytes per particle of capacity: a 32-byte placement
 * record per species, a 48-byte entry each in the accepted-pair and the
 * candidate lists, the 4-byte network output; and 40 bytes per cell), the
 * network buffers and the stats, all within cfg->mem_budget_bytes.
 * Synchronous.  EINVAL on bad sizes, ENOMEM if the budget or the device
 * cannot hold it. */
compton_status compton_init(const compton_config* cfg, struct compton_ctx** out);

/* Free everything compton_init allocated.  Synchronous.  NULL is allowed. */
compton_status compton_destroy(struct compton_ctx* ctx);

/* Text of the last CUDA error seen by this context ("" if none). */
const char* compton_last_error(const struct compton_ctx* ctx);
const char* compton_strerror(compton_status s);

/* Synchronise `stream` and report errors recorded by kernels since the last
 * check (ERANGE for a cell index outside [0, n_cells)); clears them. */
compton_status compton_check(struct compton_ctx* ctx, compton_stream_t stream);

/* Synchronise `stream`, copy the counters to *out_host and, if reset != 0,
 * zero them. */
compton_status compton_get_stats(struct compton_ctx* ctx, compton_stats* out_host, int reset,
                                 compton_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Step 1: binning and random in-cell pairing (Sec. 3.1, first step)       */
/* ---------------------------------------------------------------------- */

/* Bin both species by cell and order each cell at random: particles of a cell
 * are sorted by (key, id) with key = word 0 of Philox4x32-10 under key
 * (seed lo, seed hi) at counter (id, step lo, stream, step hi), stream 1 for
 * electrons and 2 for photons.  The order depends only on the set of
 * (cell, id) values, never on the input order or on thread timing.
 *
 * e_in/g_in are read; e_out/g_out (same n, distinct memory) receive the
 * sorted copies of all five arrays, and of the weights where the input
 * species has them (the output species then needs w_dev too).  Fills
 * *pairs_out (see compton_pairs); a pair list binned with weights on either
 * species is for compton_scatter_step on weighted species only.
 * EINVAL for null pointers, aliasing in/out, n > max_particles; a cell index
 * outside [0, n_cells) is reported by compton_check (ERANGE) and that
 * particle is left out of every cell. */
compton_status compton_bin_pairs(struct compton_ctx* ctx, const compton_species* e_in,
                                 const compton_species* g_in, compton_species* e_out,
                                 compton_species* g_out, uint64_t step,
                                 compton_pairs* pairs_out, compton_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Steps 2-3: probability, Bernoulli trial, collision (Sec. 3.1, 3.2)      */
/* ---------------------------------------------------------------------- */

/* Resolve every pair of `pairs` in place on the sorted species e, g (the
 * e_out/g_out of the compton_bin_pairs call that produced `pairs`).
 * Per pair p (cell c, density n_c = max(N_e,c, N_g,c) * w_over_v):
 *   x = gamma eps - u.k, v = 1 - beta cos(psi) (rest-frame photon energy and
 *   flux factor), s = sigma_KN(x)/sigma_T, P = 1 - exp(-n_c dt s v);
 *   u0 = (w >> 8) 2^-24 with w word p mod 4 of Philox4x32-10 at counter
 *   (p / 4, step lo, 3, step hi); collide iff u0 < P; then, from the block at
 *   (p, step lo, 4, step hi), t = 1 - cos(theta') from the Klein-Nishina
 *   angular distribution at u1 = ((r0 >> 8) + 1/2) 2^-24 and
 *   phi = 2 pi (r1 >> 8) 2^-24, and both momenta are replaced so that energy
 *   and momentum are conserved (FP64 where gamma eps exceeds the threshold).
 * Only pairs with u0 < 1 - exp(-2 n_c dt), the bound of every pair's P, are
 * evaluated (the decisions are those of evaluating all pairs); with
 * prob_out_dev given, every pair is evaluated.
 * Unequal weights (either species with w_dev): the pair's density is
 * n_p = max(N_e,c, N_g,c) * max(w_e, w_g) (P_max = 2 sigma_T c dt max w of
 * Sec. 3.2 per pair), so the expected number of real events in the cell is
 * n_e n_g sigma v dt V as with equal weights; a collision then updates the
 * lighter partner always and the heavier one only if
 * (r2 >> 8) 2^-24 < w_light / w_heavy, r2 word 2 of the angle block (weight
 * rejection: energy and momentum are conserved on average).  Equal weights
 * reduce to the unweighted step.  The species must be binned with their
 * weights (EINVAL otherwise).
 * mode selects the analytic probability or the surrogate network (the
 * paper's network takes w_e, w_g and P_max = 2 n_p dt among its inputs).
 * prob_out_dev (nullable, float[max_pairs]) receives P per pair;
 * flag_out_dev (nullable, uint8[max_pairs]) receives the decision.
 * Adds to the context stats.  ENOMODEL if a network mode has no weights. */
compton_status compton_scatter_step(struct compton_ctx* ctx, compton_species* e, compton_species* g,
                                    const compton_pairs* pairs, compton_mode mode, uint64_t step,
                                    float* prob_out_dev, uint8_t* flag_out_dev,
                                    compton_stream_t stream);

/* The same resolution on an explicit pair list (no binning): pair i is
 * (u[i], k[i]) with density n_dens_dev[i], counter id i under Philox key
 * (seed lo, seed hi).  u and k (3 SoA arrays each, length n) are updated in
 * place.  Used for pre-paired batches (serving) and for producing the
 * network's training targets. */
compton_status compton_scatter_pairs(struct compton_ctx* ctx, float* ux_dev, float* uy_dev,
                                     float* uz_dev, float* kx_dev, float* ky_dev, float* kz_dev,
                                     const float* n_dens_dev, int64_t n, uint64_t seed,
                                     uint64_t step, compton_mode mode, float* prob_out_dev,
                                     uint8_t* flag_out_dev, compton_stream_t stream);

/* No-Time-Counter collisions (Sec. 3.1, second step; Bird 1989) of the
 * binned species e, g (the e_out/g_out of the compton_bin_pairs call that
 * produced `pairs`; only its cell offsets are used), in place.  Cell c with
 * N_e, N_g > 0 draws N = floor(E + U) candidate pairs, E = N_e N_g w_over_v
 * 2 dt (2 sigma_T c bounds sigma v), U from Philox at (c, step lo, 5,
 * step hi); candidate j draws the block (c, step lo, 6 | j << 8, step hi):
 * word 0 picks the electron e_start + floor(w0 N_e / 2^32), word 1 the
 * photon, and the pair collides iff (w2 >> 8) 2^-24 < r = sigma_KN(x) v /
 * (2 sigma_T); the collision uses word 3 for the angle and word 0 of block
 * (c, step lo, 7 | j << 8, step hi) for the azimuth, and later candidates of
 * the cell see the updated momenta.  The stats count candidates as pairs
 * tested.  Analytic probability and equal weights only (EINVAL for species
 * with w_dev or a pair list binned with weights). */
compton_status compton_scatter_step_ntc(struct compton_ctx* ctx, compton_species* e, compton_species* g,
                                        const compton_pairs* pairs, uint64_t step, compton_stream_t stream);

/* Analytic target of the surrogate: r = s(x) (1 - beta cos psi) / 2 in [0, 1]
 * per pair, the probability normalised by its per-cell maximum
 * P_max = 2 sigma_T c dt max w (Sec. 3.2) in the small-probability limit.
 * Inputs u, k as in compton_scatter_pairs (read only); r_out_dev float[n]. */
compton_status compton_kn_ratio(struct compton_ctx* ctx, const float* ux_dev, const float* uy_dev,
                                const float* uz_dev, const float* kx_dev, const float* ky_dev,
                                const float* kz_dev, int64_t n, float* r_out_dev,
                                compton_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Surrogate network (Sec. 2: a network object loaded once from exported   */
/* parameters and run on any batch; Sec. 3.2: it replaces the probability */
/* calculation).  Architecture: 6 inputs, 4 hidden layers of 64 SiLU       */
/* units, 1 sigmoid output predicting r = sigma_KN v / (2 sigma_T), the    */
/* probability normalised by the cell maximum P_max = 2 sigma_T c dt max w.*/
/* Inputs f = [sgnlog(u/s_u)/n_u, sgnlog(k/s_k)/n_k], sgnlog(z) =          */
/* sign(z) ln(1 + |z|).                                                    */
/* Parameter vector (12993 floats): W0 (64x6), b0 (64), W1 (64x64), b1,    */
/* W2, b2, W3, b3, W4 (1x64), b4; each W row-major (out, in).              */
/* ---------------------------------------------------------------------- */

/* Copy the parameters from host memory (n_params must be 12993), reset the
 * Adam moments, and build the BF16 / FP8 / FP32 weight images the kernels
 * read.  feature_scales_host (nullable) = {s_u, n_u, s_k, n_k}, all > 0;
 * default {1, 7, 1e-4, 10}.  Synchronous. */
compton_status compton_mlp_set_params(struct compton_ctx* ctx, const float* theta_host, int64_t n_params,
                                      const float* feature_scales_host);

/* Copy the current FP32 parameters to host memory.  Synchronous. */
compton_status compton_mlp_get_params(struct compton_ctx* ctx, float* theta_host, int64_t n_params);

/* Set the FP8 per-tensor activation scales from a calibration batch: the
 * input of each hidden layer is stored as E4M3(h * 448 / max|h|) with the
 * maxima measured by an FP32 forward pass over the n pairs given. */
compton_status compton_mlp_calibrate(struct compton_ctx* ctx, const float* ux_dev, const float* uy_dev,
                                     const float* uz_dev, const float* kx_dev, const float* ky_dev,
                                     const float* kz_dev, int64_t n, compton_stream_t stream);

/* r_out_dev[i] = network(u[i], k[i]) for i < n, in the precision `mode`
 * selects (MLP_FP32: CUDA cores; MLP_BF16, MLP_FP8: tensor cores with FP32
 * accumulation).  ENOMODEL before compton_mlp_set_params / load. */
compton_status compton_mlp_infer(struct compton_ctx* ctx, const float* ux_dev, const float* uy_dev,
                                 const float* uz_dev, const float* kx_dev, const float* ky_dev,
                                 const float* kz_dev, int64_t n, compton_mode mode, float* r_out_dev,
                                 compton_stream_t stream);

/* One Adam step of the network on a minibatch (Sec. 3.2: mean absolute error
 * loss, Adam optimizer): inputs u, k (device SoA, length n), targets y_dev
 * (the analytic r, e.g. from compton_kn_ratio), per-sample weights w_dev
 * (nullable = 1; the data balancing of Sec. 3.2), learning rate lr.
 * Loss L = sum w |y' - y| / sum w with the subgradient 0 at y' = y; Adam with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-7 on the FP32 master parameters; the
 * BF16 / FP8 / FP32 inference images are rebuilt after the step.
 * loss_out_host (nullable): if given, the call synchronises and stores the
 * loss of this minibatch (before the update).  ERANGE if n > max_train_batch. */
compton_status compton_mlp_train_step(struct compton_ctx* ctx, const float* ux_dev, const float* uy_dev,
                                      const float* uz_dev, const float* kx_dev, const float* ky_dev,
                                      const float* kz_dev, const float* y_dev, const float* w_dev, int64_t n,
                                      float lr, float* loss_out_host, compton_stream_t stream);

/* Arithmetic of the following compton_mlp_train_step calls (Sec. 3.2
 * trains the network; the precision is this library's choice).
 * COMPTON_MODE_MLP_FP32 (the default): forward and backward in FP32 on the
 * CUDA cores, one sample per thread.  COMPTON_MODE_MLP_BF16: every
 * contraction (forward z = a W^T, backward delta W and the weight gradients
 * delta^T a) on the tcgen05 tensor cores with BF16 operands and FP32
 * accumulation in tensor memory, 128-sample tiles, one CTA per SM holding all
 * 512 TMEM columns; pre-activations, bias and output-layer gradients, the
 * loss and Adam stay in FP32.  Both compute the same gradient (the loss
 * normalised by sum w) to within BF16 rounding.  EINVAL for another mode. */
compton_status compton_mlp_set_train_precision(struct compton_ctx* ctx, compton_mode mode);

/* Data-balancing weights (Sec. 3.2: events of every probability range
 * should appear about equally often in training).  Sample i falls in bin
 * b = number of edges_host[1 .. n_bins-1] that are <= r_dev[i] (values beyond
 * the outer edges go to the outer bins); w_out_dev[i] = n / (count_b *
 * number of non-empty bins), so the weights average to 1 and each non-empty
 * bin carries equal total weight.  edges_host: n_bins + 1 strictly
 * increasing floats (host), 1 <= n_bins <= 256. */
compton_status compton_mlp_balance_weights(struct compton_ctx* ctx, const float* r_dev, int64_t n,
                                           const float* edges_host, int32_t n_bins, float* w_out_dev,
                                           compton_stream_t stream);

/* The gradient dL/dtheta of the last compton_mlp_train_step (the loss
 * normalised by sum w), same layout as the parameters.  Synchronous. */
compton_status compton_mlp_get_grad(struct compton_ctx* ctx, float* grad_host, int64_t n_params);

/* Select the network's inputs for every later inference, calibration and
 * training step.  COMPTON_FEATURES_MOMENTA (the default) feeds the six
 * sgnlog-scaled momentum components, as the paper feeds momenta (Sec. 3.2).
 * COMPTON_FEATURES_INVARIANTS (no counterpart in the paper: an ablation of
 * that choice) feeds f0 = ln(x)/8 and f1 = ln(v)/8, with x the photon energy
 * in the electron rest frame and v = 1 - beta cos psi from the FP32
 * invariants, and zeros in the other four inputs; the network must then be
 * trained in that mode.  EINVAL for another value. */
compton_status compton_mlp_set_features(struct compton_ctx* ctx, int32_t features);

/* The network's training range: pairs with gamma > gamma_max or eps outside
 * [eps_min, eps_max] take the analytic probability instead (and are counted
 * as fallbacks).  Default gamma_max = 1e3, eps in [1e-4, 1].  Saved with the
 * network.  EINVAL unless 1 <= gamma_max, 0 <= eps_min < eps_max, finite. */
compton_status compton_mlp_set_range(struct compton_ctx* ctx, double gamma_max, double eps_min, double eps_max);

/* Serialise the network (format "CMLP" version 3: header with the Adam step,
 * feature scales and mode, training range, activation scales, then parameters
 * and both Adam moments; version 1 and 2 blobs still load, keeping the
 * context's mode or range where they carry none) to buf.  With buf NULL,
 * *len receives the size needed; ERANGE if *len is too small.
 * Synchronous. */
compton_status compton_mlp_save(struct compton_ctx* ctx, void* buf, size_t* len);

/* Load a blob written by compton_mlp_save.  EINVAL on a bad header or size. */
compton_status compton_mlp_load(struct compton_ctx* ctx, const void* buf, size_t len);

/* ---------------------------------------------------------------------- */
/* The paper's own network (Sec. 3.2, Fig. 2a): 9 inputs, hidden layers of */
/* 9, 12 and 9 ReLU units, one sigmoid output; 337 FP32 parameters.        */
/* ---------------------------------------------------------------------- */

#define COMPTON_PNET_PARAMS 337

/* Load the parameters theta (host, 337 floats, layer by layer: W0 (9 x 9),
 * b0 (9), W1 (12 x 9), b1 (12), W2 (9 x 12), b2 (9), W3 (1 x 9), b3 (1), each
 * W (out, in) row-major), reset the Adam state, and set the feature scales
 * (host, 4 floats s_u, n_u, s_k, n_k, all > 0; NULL keeps the current ones,
 * by default 1, 7, 1e-4, 10) and the training range (as for
 * compton_mlp_set_range).  Inputs of a pair:
 *   sgnlog(u_i / s_u) / n_u, sgnlog(k_i / s_k) / n_k   (i = x, y, z),
 *   ln(w_e) / 8, ln(w_g) / 8, ln(P_max) / 8,
 * sgnlog(z) = sign(z) ln(1 + |z|), w the macro-particle weight over the cell
 * volume, P_max = 2 n dt the cell's probability bound (sigma_T c = 1); output
 * r = sigma_KN v / (2 sigma_T).  After this call COMPTON_MODE_PNET is
 * available to the scatter step, which gives both species the context's
 * w_over_v.  EINVAL on a wrong count, scale or range.  Synchronous. */
compton_status compton_pnet_set_params(struct compton_ctx* ctx, const float* theta_host, int64_t n_params,
                                       const float* feature_scales_host, double gamma_max, double eps_min,
                                       double eps_max);

/* Copy the parameters and / or the gradient of the last train step (the loss
 * normalised by sum w) to the host (either pointer may be NULL).  ENOMODEL
 * before compton_pnet_set_params.  Synchronous. */
compton_status compton_pnet_get_params(struct compton_ctx* ctx, float* theta_host, float* grad_host,
                                       int64_t n_params);

/* r for n explicit pairs (device SoA momenta, device r_out[n]) at the given
 * weights and P_max (all > 0).  Asynchronous on stream. */
compton_status compton_pnet_infer(struct compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                  const float* kx, const float* ky, const float* kz, int64_t n, float w_e,
                                  float w_g, float p_max, float* r_out, compton_stream_t stream);

/* One Adam step (beta 0.9, 0.999, epsilon 1e-7) on the weighted mean absolute
 * error sum_i w_i |y'_i - y_i| / sum_i w_i over n > 0 device samples (targets
 * y, weights w, NULL = all 1); the ReLU and |.| subgradients at 0 are 0.  With
 * loss_out_host non-NULL the step's loss (before the update) is written there
 * and the call synchronises on stream; else it is asynchronous. */
compton_status compton_pnet_train_step(struct compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                       const float* kx, const float* ky, const float* kz, const float* y,
                                       const float* w, int64_t n, float w_e, float w_g, float p_max, float lr,
                                       float* loss_out_host, compton_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of pre-paired batches (Sec. 2: the network */
/* object runs "for any given batch of inputs"; a PIC code produces such   */
/* batches from many tiles and time steps).                                */
/* ---------------------------------------------------------------------- */

/* One request: n pre-paired electrons/photons (device arrays, read), the
 * arrays that receive the momenta after the step (device, may equal the
 * inputs), the pair density per pair (n_dens_dev, nullable) or one value
 * (n_dens), the request's Philox seed and step, and the probability mode.
 * Pair i of a request uses counter id i under key seed, exactly as
 * compton_scatter_pairs, so its result does not depend on what else runs. */
typedef struct compton_request {
    const float* ux_in_dev;
    const float* uy_in_dev;
    const float* uz_in_dev;
    const float* kx_in_dev;
    const float* ky_in_dev;
    const float* kz_in_dev;
    float* ux_out_dev;
    float* uy_out_dev;
    float* uz_out_dev;
    float* kx_out_dev;
    float* ky_out_dev;
    float* kz_out_dev;
    const float* n_dens_dev;
    float n_dens;
    int64_t n;
    uint64_t seed;
    uint64_t step;
    compton_mode mode;
} compton_request;

typedef struct compton_result {
    compton_status status;
    uint64_t scatters;  /* collisions in this request                      */
    double latency_s;   /* from compton_submit to completion (host clock)  */
    double queue_s;     /* from compton_submit to admission                */
} compton_result;

/* Start the serving engine: a device pool of pool_bytes (the memory budget;
 * each admitted request holds 28 bytes per pair, 32 in surrogate modes) and
 * at most max_active requests admitted at once.  The pool is allocated here,
 * once.  EINVAL if already started. */
compton_status compton_serve_start(struct compton_ctx* ctx, uint64_t pool_bytes, int32_t max_active);

/* Stop the engine after the work in flight; requests not yet done are
 * dropped.  compton_destroy calls it. */
compton_status compton_serve_stop(struct compton_ctx* ctx);

/* Queue a request; returns at once with a ticket.  The engine admits it when
 * a block of the pool fits it and runs its tiles together with the other
 * admitted requests.  The caller keeps the input and output arrays alive and
 * unchanged until compton_poll returns OK.  ERANGE if the request can never
 * fit the pool, EBUSY if the queue is full (retry), ENOMODEL for a surrogate
 * mode without a network.  Thread-safe. */
compton_status compton_submit(struct compton_ctx* ctx, const compton_request* req, uint64_t* ticket);

/* ENOTREADY until the request's outputs are written, then OK with *out
 * filled (the ticket is retired).  EINVAL for an unknown ticket.
 * Thread-safe. */
compton_status compton_poll(struct compton_ctx* ctx, uint64_t ticket, compton_result* out);

/* Pool bytes in use now, the peak since start, and the pool size. */
compton_status compton_serve_info(struct compton_ctx* ctx, uint64_t* bytes_in_use, uint64_t* peak_bytes,
                                  uint64_t* pool_bytes);

/* Per-cell offsets of one species with no device allocation at all (the
 * paper has no counterpart: this serves callers that cannot allocate device
 * memory when they need the offsets, such as a particle-in-cell code whose
 * memory manager owns all device memory, or a time-step loop that must not
 * allocate).  cell_dev: n int32 cell indices (device); off_out_dev: n_cells
 * + 1 int32 (device, caller-owned).  off_out_dev[c] = number of particles
 * with a cell index below c; off_out_dev[n_cells] = the number counted.
 * Indices outside [0, n_cells) are skipped without an error (unlike
 * compton_bin_pairs, which reports them through compton_check): the caller
 * sees how many were skipped as n - off_out_dev[n_cells].  For in-range input
 * these are the values of compton_pairs.off_*_dev of compton_bin_pairs.
 * Needs no context.  The counts live in a library-owned static device array
 * of 2^20 int32 plus 256 strip sums (about 4 MiB, held on every GPU that
 * loads the library until exit): n_cells above 1048576 is rejected with
 * ERANGE, n < 0 or above INT32_MAX with EINVAL.  The first call on a device
 * looks up that array's device address (and the SM count), so make it before
 * any stream capture; a cudaDeviceReset makes the kept address stale, so do
 * not call this after a reset in the same process.  Every call reuses the
 * array and clears it first; calls whose work overlaps on the GPU race on it
 * and must be ordered by the caller.  An error pending from the caller's
 * earlier work is cleared on entry and not reported as this call's; ECUDA
 * means a launch of this call failed.  Asynchronous on `stream`. */
compton_status compton_cell_offsets_noalloc(const int32_t* cell_dev, int64_t n, int64_t n_cells,
                                            int32_t* off_out_dev, compton_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Per-kernel timing (measurement support; no counterpart in the paper).   */
/* ---------------------------------------------------------------------- */

/* Kernel slots of compton_kernel_times. */
typedef enum compton_kernel_slot {
    COMPTON_K_COUNT = 0,   /* histogram and order check                    */
    COMPTON_K_SCAN = 1,    /* the three scan kernels together              */
    COMPTON_K_PLACE = 2,   /* keyed placement (shuffled input)             */
    COMPTON_K_SORT = 3,    /* per-cell sort and sorted copy                */
    COMPTON_K_PROB = 4,    /* probability and Bernoulli trial of all pairs */
    COMPTON_K_COLLIDE = 5, /* collisions of the accepted pairs             */
    COMPTON_K_MLP = 6,     /* surrogate network forward                    */
    COMPTON_K_NTC = 7,     /* No-Time-Counter candidates and collisions    */
    COMPTON_N_TIMED = 8
} compton_kernel_slot;

/* enable != 0: from now on every kernel launch of the slots above records a
 * CUDA event pair on its own stream (the last 64 launches per slot are kept)
 * and the counts restart from zero; enable == 0 stops recording.  The events
 * are created on the first enable.  Synchronous.  ECUDA if they cannot be
 * created. */
compton_status compton_kernel_timing(struct compton_ctx* ctx, int32_t enable);

/* Wait for the recorded events and write, per slot, the summed device time
 * of the kept launches in ms (ms_out_host[COMPTON_N_TIMED]) and their number
 * (launches_out_host[COMPTON_N_TIMED]).  EINVAL if timing was never enabled. */
compton_status compton_kernel_times(struct compton_ctx* ctx, double* ms_out_host, int64_t* launches_out_host);

/* Self-test of the give-up path of the bounded device waits (every wait of
 * the tensor-core kernels is limited in time; on expiry the kernel records a
 * timeout, frees its tensor memory and returns instead of hanging): one
 * thread waits on a barrier that nothing completes, for timeout_ns
 * (<= 10 s).  compton_check then returns ETIMEOUT.  The paper has no
 * counterpart; this exists so the failure path can be tested without a
 * fault. */
compton_status compton_selftest_wait(struct compton_ctx* ctx, uint64_t timeout_ns, compton_stream_t stream);

/* Host-side fault injection, for testing the error paths (the paper has no
 * counterpart).  Process-wide: after this call the library's checks of CUDA
 * calls let `skip` of them pass and then report `fail` failures, without
 * making the failing call and without touching the device: the device
 * allocation of compton_init and compton_serve_start then fails as if out of
 * memory (ENOMEM), any other checked call or launch as a CUDA error (ECUDA,
 * with compton_last_error naming the call).  fail = 0 disarms it.
 * pending_out (nullable): failures still pending from the previous arming.
 * The context stays usable after an injected failure: the next call of the
 * same entry point starts from a clean state.  EINVAL for negative counts. */
compton_status compton_debug_inject(int64_t skip, int64_t fail, int64_t* pending_out);

/* The scattering-angle sampler of compton_scatter_step on its own, for
 * validation (the paper resolves each collision by sampling the scattered
 * photon, Sec. 3.1).  For each i: x_dev[i] is the rest-frame photon energy,
 * r_dev[i] a raw 32-bit random word (its top 24 bits give
 * u1 = ((r >> 8) + 1/2) 2^-24); the outputs are cos(theta'), sin(theta') of
 * the inverse of the Klein-Nishina angular cumulative at u1, and the Compton
 * energy ratio 1/(1 + x (1 - cos theta')).  All arrays length n, device. */
compton_status compton_kn_sample_angle(struct compton_ctx* ctx, const float* x_dev, const uint32_t* r_dev,
                                       int64_t n, float* cth_out_dev, float* sth_out_dev,
                                       float* ratio_out_dev, compton_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* COMPTON_H */
