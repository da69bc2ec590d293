/*
 * tcw.h -- C ABI of the GB300 (sm_103a) long-transient track-statistic search.
 *
 * The method is the template-bank search of Merou, Tenorio & Sintes,
 * "GPU-Accelerated Searches for Long-Transient Gravitational Waves from
 * Newborn Neutron Stars" (arXiv:2507.07816):
 *
 *   Eq. 1  f(t)    = f0 * ((t - T0)/tau + 1)^(1/(1-n))          (Sec. 1)
 *   Eq. 2  fhat(t) = f(t) * (1 + v(t).nhat / c)                  (Sec. 1)
 *   Sec. 2 each template selects one bin per SFT segment; the weighted
 *          normalized power is summed over the selected bins:
 *          S = sum w rho,  W1 = sum w,  W2 = sum w^2
 *   Eq. 4  Psi = (S - <S>)/sigma_S = (S - W1)/sqrt(W2)
 *
 * Readings of points the paper leaves open, used throughout this library:
 *   - bin k has centre f_min + k*df; the track takes the nearest centre,
 *     k = floor((fhat - f_min)/df + 1/2);
 *   - segments with t_mid < T0 and lookups with k outside [0, n_bin) add
 *     nothing to S, W1 or W2;
 *   - detectors are summed into one statistic; Psi = -inf when W2 == 0;
 *   - top-k per sky orders by (Psi descending, caller template index
 *     ascending).
 *
 * Conventions for every entry point:
 *   - Return value: TCW_OK (0) or a negative tcw_status; no call aborts or
 *     exits.  tcw_status_string() names a code; tcw_last_error() returns a
 *     human-readable message for the most recent failure on a context.
 *   - Arrays are dense, C order (last index fastest), in the element type
 *     named in the declaration.
 *   - Pointer flags: TCW_HOST (0) means host memory; TCW_DEVICE (1) means
 *     device memory on the context's device.  Host inputs are copied into
 *     buffers the context owns before the call returns.  Device inputs are
 *     copied too (device to device), so the caller may free them after the
 *     call returns.  Outputs are caller-allocated.
 *   - Thread safety: one context per host thread.  All device work of a
 *     context runs on its stream, in call order.
 */
#ifndef TCW_H
#define TCW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tcw_ctx tcw_ctx;
typedef int tcw_status;

enum {
    TCW_OK = 0,
    TCW_ERR_INVALID_ARGUMENT = -1, /* bad size, pointer, value or flag */
    TCW_ERR_CUDA = -2,             /* a CUDA runtime call failed */
    TCW_ERR_OUT_OF_MEMORY = -3,    /* device allocation failed */
    TCW_ERR_STATE = -4,            /* a required input has not been loaded */
    TCW_ERR_UNSUPPORTED = -5,      /* inputs outside what the kernels handle */
    TCW_ERR_DEVICE = -6,           /* a kernel reported an internal error */
    TCW_ERR_TIMEOUT = -7           /* a bounded device wait ran out */
};

enum { TCW_HOST = 0, TCW_DEVICE = 1 };
enum { TCW_F32 = 0, TCW_F16 = 1 };

/* Search kernels.  TCW_KERNEL_AUTO picks the group kernel when its exactness
 * conditions hold and the per-lookup kernel otherwise. */
enum {
    TCW_KERNEL_AUTO = 0,
    TCW_KERNEL_GROUP = 1,   /* sky-group candidate-pair kernel (fast path) */
    TCW_KERNEL_LOOKUP = 2   /* one thread per (sky, template), FP64 per lookup */
};

/* Options for tcw_set_option. */
enum {
    TCW_OPT_KERNEL = 1,        /* one of TCW_KERNEL_* */
    TCW_OPT_KEEP_STATS = 2,    /* 1: keep S, W1, W2 of the last search for
                                  tcw_get_statistics (costs 3*4 B per pair) */
    TCW_OPT_TILE_SEGMENTS = 3, /* segments per tile of the group kernel: the spacing of
                                  the FP64 track anchors and of the fp32 partial sums;
                                  a power of two in [8, 128], default 32 */
    TCW_OPT_BANK_CHUNK = 4,    /* template groups of one pass (1024/lanes sorted
                                  templates) per work item of the group kernel,
                                  in [1, 4096], default 1 */
    TCW_OPT_AUTOTUNE = 5,      /* batched search: 1 (default) = choose the bank chunk
                                  and tile length by timing candidates on a sample of
                                  the batch; 0 = use TCW_OPT_BANK_CHUNK and
                                  TCW_OPT_TILE_SEGMENTS */
    TCW_OPT_BATCH_MEMORY = 6,  /* batched search: bytes of Psi and anchor buffers per
                                  wave of events (default 48 GiB, minimum 1 MiB) */
    TCW_OPT_SKY_LANES = 7,     /* sky groups of 16 per chunk of the group kernel: 16,
                                  32 or 64 (a pass covers 16*lanes skies x 1024/lanes
                                  templates); 0 (default) = the lowest cost for the
                                  sky count, the bank size and the SM count */
    TCW_OPT_TRIAGE_SPREAD = 8, /* triaged search: a chosen patch suppresses the patches
                                  within this many positions (default 2; 0 = plain
                                  ranking); best suppressed ones fill up if needed */
    TCW_OPT_AMPLITUDE_POWER = 9, /* p in [0, 8]: every lookup's weight w_{d,j} is
                                  multiplied by the template's own amplitude
                                  weight (f(t_j)/f0)^p, so S, W1 = sum w and
                                  W2 = sum w^2 of Eq. 4 use w_{d,j} (f(t_j)/f0)^p.
                                  The signal power grows as h0^2 and h0 as f^2
                                  (Eq. 3 of arXiv:2507.07816), so p = 4 weights
                                  each segment by the expected signal power of
                                  the template; default 0 (the weights as given).
                                  Applies to tcw_search, tcw_search_batched and
                                  the exhaustive part of tcw_search_triaged */
    TCW_OPT_GEN_CHUNK = 10,    /* tcw_search_generated: templates per chunk, a multiple
                                  of 64 in [64, 2^24] (default 2^18) */
    TCW_OPT_TRACK_BINS = 11,   /* bins per lookup: 1 (default) = the nearest bin, as
                                  in the paper; 2 = the two bins whose centres
                                  bracket the track, k = floor((fhat - f_min)/df)
                                  and k + 1, both required in the band, their
                                  powers (or counts) summed; Eq. 4 then uses twice
                                  the mean and variance (independent bins).  For
                                  tracks between bins or moving more than a bin per
                                  SFT, whose power leaks into the neighbour.
                                  tcw_track_bins reports k.  Applies like
                                  TCW_OPT_AMPLITUDE_POWER, and to
                                  tcw_search_generated */
    TCW_OPT_TRIAGE_TEMPLATES = 12 /* triaged search: parameter regions too.  Per
                                  mille of the bank searched at each chosen patch:
                                  the templates with the highest coarse Psi at that
                                  patch's representative sky; the union over the
                                  chosen patches is searched at all their skies.
                                  In [1, 1000], default 1000 (every template) */,
    TCW_OPT_TRIAGE_STRIDE = 13 /* triage coarse pass: use every stride-th segment
                                  (segments 0, s, 2s, ...) for the coarse Psi and its
                                  features; in [1, 64], default 1 (every segment) */
};

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on, or NULL for a stream the context creates and owns.
 * Errors: INVALID_ARGUMENT (out == NULL, bad device), CUDA. */
tcw_status tcw_create(tcw_ctx **out, int device, void *cuda_stream);

/* Free every device buffer and the owned stream.  NULL is accepted. */
tcw_status tcw_destroy(tcw_ctx *ctx);

/* Set an option (TCW_OPT_*).  Errors: INVALID_ARGUMENT. */
tcw_status tcw_set_option(tcw_ctx *ctx, int option, int64_t value);

/* Statistic summed along the tracks (Sec. 2 of arXiv:2507.07816 names two):
 *   TCW_STAT_POWER          s = sum w rho; Eq. 4 with <s> = W1, sigma^2 = W2
 *                           (default; rho_th ignored)
 *   TCW_STAT_NUMBER_COUNT   s = sum w nu with nu = 1 where the bin's power
 *                           exceeds rho_th strictly (compared in double),
 *                           else 0; under noise rho ~ Exp(1), so nu is
 *                           Bernoulli(q), q = exp(-rho_th), and Eq. 4 uses
 *                           <s> = q W1, sigma^2 = q (1 - q) W2.
 * The spectrogram stays loaded as power; the count is taken from it on the
 * device (a bit map of n_det x n_seg x (n_bin/32 + 2) words, rebuilt after
 * each load or threshold change).  Applies to tcw_search, tcw_search_batched,
 * tcw_search_triaged (its exhaustive part; the coarse ranking stays on power)
 * and tcw_statistics (S = sum w nu).  Not available in tcw_search_noalloc.
 * Errors: INVALID_ARGUMENT (unknown statistic; rho_th not finite and > 0). */
enum { TCW_STAT_POWER = 0, TCW_STAT_NUMBER_COUNT = 1 };
tcw_status tcw_set_statistic(tcw_ctx *ctx, int statistic, double rho_th);

/*
 * Load the normalized-power spectrogram (Sec. 2: SFT data processed into
 * normalized power rho_j) of n_det detectors that share segment times.
 *   rho      [n_det][n_seg][n_bin], dtype TCW_F32 (float) or TCW_F16 (IEEE
 *            half); bin k of segment j has centre f_min + k*df.
 *   t_mid    [n_seg] segment mid-times (s), strictly increasing, finite.
 *   weights  [n_det][n_seg] float, finite and >= 0 (the antenna-pattern and
 *            noise-floor weights of Sec. 2), or NULL for all ones.
 *   rho_flags applies to rho; t_mid and weights are always host pointers.
 * Replaces any previous spectrogram and invalidates the loaded velocities
 * when n_det or n_seg change.
 * Errors: INVALID_ARGUMENT (sizes < 1, n_bin > 2^30, df <= 0, non-finite
 * f_min, unsorted t_mid, bad weights, NULL), OUT_OF_MEMORY, CUDA. */
tcw_status tcw_load_spectrogram(tcw_ctx *ctx, int n_det, int64_t n_seg, int64_t n_bin,
                                int dtype, const void *rho, int rho_flags,
                                double f_min, double df, const double *t_mid,
                                const float *weights);

/*
 * Load detector velocities relative to the solar-system barycentre (Eq. 2),
 *   v [n_det][n_seg][3] double, m/s, same frame as the sky vectors.
 * Errors: STATE (no spectrogram), INVALID_ARGUMENT (NULL, non-finite,
 * |v| >= c/100), CUDA. */
tcw_status tcw_load_velocity(tcw_ctx *ctx, const double *v, int flags);

/*
 * Define the template bank (Eq. 1 parameters), [n_tmpl] doubles each:
 * f0 > 0 (Hz), tau > 0 (s), n > 1 (Eq. 1 is singular at n = 1); and the
 * signal start time T0 (s), shared by the bank.
 * Errors: INVALID_ARGUMENT (n_tmpl < 1, n_tmpl > 2^31 - 1, NULL, a value out
 * of range or non-finite), OUT_OF_MEMORY, CUDA. */
tcw_status tcw_define_bank(tcw_ctx *ctx, int64_t n_tmpl, const double *f0,
                           const double *tau, const double *n, double T0, int flags);

/*
 * Define the sky directions: nhat [n_sky][3] double unit vectors toward the
 * source (|nhat| within 1e-9 of 1).
 * Errors: INVALID_ARGUMENT (n_sky < 1, NULL, non-unit), OUT_OF_MEMORY, CUDA. */
tcw_status tcw_define_sky(tcw_ctx *ctx, int64_t n_sky, const double *nhat, int flags);

/*
 * Run the search (track, Doppler, bin, gather, weighted sum, Psi, top-k) and
 * write, per sky s in caller order, the k best templates:
 *   psi_out [n_sky][k] float   Psi, descending
 *   idx_out [n_sky][k] int64   caller template index (ties: ascending index)
 * 1 <= k <= min(n_tmpl, 1024).  out_flags: TCW_HOST or TCW_DEVICE for both
 * outputs.  The call returns after the device work has finished.
 * Errors: STATE (missing spectrogram, velocity, bank or sky),
 * INVALID_ARGUMENT, UNSUPPORTED (explicit group kernel requested but its
 * exactness conditions fail), DEVICE, OUT_OF_MEMORY, CUDA. */
tcw_status tcw_search(tcw_ctx *ctx, int k, float *psi_out, int64_t *idx_out, int out_flags);

/*
 * Statistics of the last search, [n_sky][n_tmpl] float in caller order (any
 * pointer may be NULL): S, W1, W2 need TCW_OPT_KEEP_STATS = 1 during the
 * search; psi is always available.
 * Errors: STATE (no search, or stats not kept), INVALID_ARGUMENT, CUDA. */
tcw_status tcw_get_statistics(tcw_ctx *ctx, float *S_out, float *W1_out, float *W2_out,
                              float *psi_out, int out_flags);

/*
 * Bin index chosen by the search kernel for every lookup, written by the
 * same kernel code with recording switched on:
 *   bins_out [n_sky][n_tmpl][n_det][n_seg] int32, caller order, -1 where the
 *   segment precedes T0 or the bin lies outside [0, n_bin).
 * Meant for small problems (the output has n_sky*n_tmpl*n_det*n_seg entries).
 * Errors: STATE, INVALID_ARGUMENT (output larger than 2^31 entries), CUDA. */
tcw_status tcw_track_bins(tcw_ctx *ctx, int32_t *bins_out, int out_flags);

/*
 * Search without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- for example
 * an application whose device memory is wholly owned by its own arena or
 * caching allocator, a real-time pipeline that cannot accept the implicit
 * device synchronisation of cudaMalloc/cudaFree, or a plug-in host that
 * forbids device allocation.
 *
 * It runs the same Doppler-table, group and top-k kernels as tcw_search, on
 * caller-owned DEVICE inputs and outputs, with no context:
 *   rho [n_det][n_seg][n_bin] (dtype TCW_F32 or TCW_F16), t_mid [n_seg]
 *   (strictly increasing), weights [n_det][n_seg] float or NULL for ones,
 *   v [n_det][n_seg][3] (m/s), f0/tau/n [n_tmpl], nhat [n_sky][3] unit
 *   vectors, psi_out/idx_out [n_sky][k] (caller order, ties by ascending
 *   template index); all on the current CUDA device; work is queued on
 *   cuda_stream (NULL = legacy default stream) and the call returns after it
 *   has finished.
 * Every intermediate buffer comes from one fixed device array of 64 MiB
 * inside the library (held by each GPU on which the library's device code is
 * loaded, until the process exits).  The intermediates take about
 *   4 Spad Bpad + 5 n_det n_seg Spad + 28 Bpad + 28 Spad + 131072 n_SM bytes
 * (+ 4 n_det n_seg when weights is NULL), with Spad = n_sky rounded up to
 * the sky chunk tcw_search picks (256, 512 or 1024 skies), Bpad = n_tmpl
 * rounded up to a multiple of 64 and n_SM the device's SM count (152 on
 * GB300: 19 MiB of per-CTA scratch); problems beyond 64 MiB are rejected
 * with TCW_ERR_UNSUPPORTED.  The sky is taken in tcw_search's Doppler order
 * (sorted on the host from the middle segment's velocity of detector 0), and
 * inputs outside the group kernel's exactness conditions run the per-lookup
 * FP64 kernel, as in tcw_search.  The track is evaluated with pow per
 * (template, segment) (no anchor table).  The first call made with a given
 * device current looks up the array's device address (cudaGetSymbolAddress)
 * and caches it.  The call synchronises cuda_stream several times and reads
 * results back, so it cannot be made while that stream is being captured
 * into a graph (it then returns TCW_ERR_STATE).  All calls share the array
 * and it keeps the previous call's contents: each call clears what must
 * start at zero, and calls that overlap on the GPU (e.g. on two streams)
 * race on it.
 * Errors: INVALID_ARGUMENT (sizes, NULL, k, or element values: f0 <= 0,
 * tau <= 0, n <= 1, non-unit nhat, |v| >= c/100, bad weights, unsorted
 * t_mid), STATE (stream capture), UNSUPPORTED, DEVICE, CUDA. */
tcw_status tcw_search_noalloc(int n_det, int64_t n_seg, int64_t n_bin, int dtype, const void *rho,
                              double f_min, double df, const double *t_mid, const float *weights,
                              const double *v, int64_t n_tmpl, const double *f0, const double *tau,
                              const double *n, double T0, int64_t n_sky, const double *nhat, int k,
                              float *psi_out, int64_t *idx_out, void *cuda_stream);

/*
 * Batched search.  The paper searches one event at a time; this form runs
 * many events -- spectrograms of uneven length, each with its own segment
 * times, detector velocities, weights, signal start T0 (Eq. 1) and sky list --
 * against the context's template bank (tcw_define_bank; its T0 is not used
 * here) in one persistent group-kernel launch per wave of events, recorded
 * once as a CUDA graph and replayed by every tcw_search_batched call.
 *
 * tcw_load_events copies every event (host or device memory per `flags`)
 * into context buffers:
 *   rho [n_det][n_seg][n_bin] of `dtype`, t_mid [n_seg] strictly increasing,
 *   weights [n_det][n_seg] >= 0 or NULL for ones, velocity [n_det][n_seg][3]
 *   in m/s (|v| < c/100), nhat [n_sky][3] unit vectors (within 1e-9).
 * Errors: INVALID_ARGUMENT (names the event and the field), UNSUPPORTED
 * (n_det > 2, or a power map smaller than 64 bytes), OUT_OF_MEMORY, CUDA.
 *
 * tcw_search_batched writes, for every event in order and every sky of that
 * event in the caller's order, the top k of Psi (Eq. 4):
 *   psi_out [total_sky][k], idx_out [total_sky][k] (caller template index),
 *   total_sky = sum of the events' n_sky; ordering as in tcw_search.
 * The first call after loading (or after a bank or option change) plans the
 * batch, runs the autotuner (TCW_OPT_AUTOTUNE) and records the graph; later
 * calls with the same k only replay it.  There is no per-lookup fallback: a
 * batch outside the group kernel's exactness conditions is UNSUPPORTED.
 * Errors: STATE (no events or bank), INVALID_ARGUMENT (k, pointers, flags),
 * UNSUPPORTED, OUT_OF_MEMORY, DEVICE, CUDA. */
typedef struct {
    const void *rho;
    const double *t_mid;
    const float *weights;
    const double *velocity;
    const double *nhat;
    int64_t n_seg;
    int64_t n_sky;
    double T0;
} tcw_event;

tcw_status tcw_load_events(tcw_ctx *ctx, int n_det, int64_t n_bin, int dtype, double f_min,
                           double df, const tcw_event *events, int n_events, int flags);
tcw_status tcw_search_batched(tcw_ctx *ctx, int k, float *psi_out, int64_t *idx_out,
                              int out_flags);

/* What the last batched search ran. */
typedef struct {
    int n_events;
    int waves;                  /* group-kernel launches per search */
    int bank_chunk;             /* groups of 8 templates per work item */
    int tile_segments;          /* anchor spacing / fp32 partial-sum length */
    int autotuned;              /* 1 if the two above came from the autotuner */
    int n_candidates;           /* shapes timed by the autotuner */
    int n_items;                /* work items over all waves */
    int graph_kernels;          /* kernel nodes in the replayed graph */
    int64_t total_sky;
    int64_t lookups;            /* sum over events of n_sky * n_tmpl * n_det * n_seg */
    int64_t general_path_lanes;
    double tune_ms;             /* host wall time of the autotuner */
    double best_rate;           /* sums/s of the winning shape on the autotuner's sample */
    double default_rate;        /* sums/s of bank_chunk 1, tile 32 on the same sample */
    double quantum;             /* fixed-point step of the Doppler factor */
    float search_ms;            /* device time of the last graph replay, ms */
} tcw_batch_info;

tcw_status tcw_get_batch_info(tcw_ctx *ctx, tcw_batch_info *info);

/* The autotuner's measurements: up to max_results (bank_chunk, tile_segments,
 * sums/s) rows; *n_results = rows available.  Errors: STATE, INVALID_ARGUMENT. */
tcw_status tcw_get_tune_results(tcw_ctx *ctx, int max_results, int *bank_chunk,
                                int *tile_segments, double *sums_per_s, int *n_results);

/*
 * Learned sky triage.  The paper has no learned component: the triage is an
 * addition that ranks sky patches so that the exhaustive search (Sec. 2,
 * Eq. 4) runs on the best-ranked ones only.
 *
 * A patch is a run of patch_size consecutive skies in the search's
 * Doppler-sorted order (v_0(t_m).nhat, t_m = the middle segment of detector
 * 0, ties by caller index); its representative is its middle sky.  The
 * coarse pass computes Psi of every template at every representative, and
 * the features of a patch are log(1 + count) over a 128-bin histogram of
 * those Psi on [psi_lo, psi_hi) (lower values and -inf in bin 0, higher ones
 * in bin 127).
 *
 * The network is an MLP 128 -> 256 -> 256 -> 1 with ReLU after both hidden
 * layers: y = relu(relu(X W1 + b1) W2 + b2) w3 + b3.  Its parameters are one
 * packed float32 vector theta[TCW_MLP_PARAMS]:
 *   W1 [128][256] | b1 [256] | W2 [256][256] | b2 [256] | w3 [256] | b3
 * and the forward pass reads the weights as bfloat16, wbf[TCW_MLP_WEIGHTS]:
 *   W1 | W2 | w3 (same element order), with fp32 accumulation.
 * The tcw_mlp_* calls take DEVICE pointers on the current device, queue work
 * on `stream` (NULL = legacy default stream) and return without waiting.
 */
#define TCW_MLP_PARAMS 99073
#define TCW_MLP_WEIGHTS 98560

/* wbf = bfloat16(theta weights), round to nearest even. */
tcw_status tcw_mlp_pack(const float *theta, uint16_t *wbf, void *stream);
/* X [n][128] -> H1 [n][256], H2 [n][256] (post-ReLU), y [n]. */
tcw_status tcw_mlp_forward(const uint16_t *wbf, const float *theta, const float *X, int64_t n,
                           float *H1, float *H2, float *y, void *stream);
/* Gradient of a loss with dL/dy = dy into grad[TCW_MLP_PARAMS] (packed like
 * theta; taken at the bfloat16 weights the forward pass used).
 * work: 2 * n * 256 floats of scratch. */
tcw_status tcw_mlp_backward(const uint16_t *wbf, const float *X, int64_t n, const float *H1,
                            const float *H2, const float *dy, float *grad, float *work,
                            void *stream);
/* Mean binary cross-entropy with logits: loss[0] = mean(pw*l*softplus(-y) +
 * (1-l)*softplus(y)), dy = its derivative in y. */
tcw_status tcw_mlp_bce(const float *y, const float *label, int64_t n, float pos_weight,
                       float *loss, float *dy, void *stream);
/* One Adam step (step counts from 1, bias-corrected) on theta with moments
 * m, v; refreshes wbf from the new theta. */
tcw_status tcw_mlp_adam(float *theta, float *m, float *v, const float *grad, int64_t step,
                        float lr, float beta1, float beta2, float eps, uint16_t *wbf,
                        void *stream);

/* Coarse pass of the loaded search (on the segments 0, s, 2s, ... with s =
 * TCW_OPT_TRIAGE_STRIDE): feat_out [n_patch][128] float32,
 * n_patch = ceil(n_sky / patch_size); psi_out [n_patch][n_tmpl] (caller
 * template order) may be NULL.  Errors: STATE, INVALID_ARGUMENT (patch_size
 * < 1, psi_hi <= psi_lo), UNSUPPORTED (more than 2 detectors, or a Doppler
 * shift above 2.9 bins), CUDA. */
tcw_status tcw_triage_features(tcw_ctx *ctx, int patch_size, float psi_lo, float psi_hi,
                               float *feat_out, float *psi_out, int out_flags);

/* Triaged search: coarse pass, network score per patch, the ceil(frac *
 * n_patch) best patches (spread apart by TCW_OPT_TRIAGE_SPREAD) searched
 * exhaustively as tcw_search does, over every template or, with
 * TCW_OPT_TRIAGE_TEMPLATES < 1000, over the union of each chosen patch's best
 * templates by coarse Psi (then a row's entries are the best of that union).
 * psi_out/idx_out [n_sky][k] as tcw_search for searched skies (caller
 * template indices); rows of skipped skies hold -inf and -1, and so do the
 * entries past the union's size when it holds fewer than k templates.
 * searched_out [n_sky] (may be NULL): 1 for searched skies.  wbf and theta
 * are device pointers.
 * Errors: as tcw_search and tcw_triage_features, INVALID_ARGUMENT (frac not
 * in (0, 1]). */
tcw_status tcw_search_triaged(tcw_ctx *ctx, const uint16_t *wbf, const float *theta,
                              int patch_size, float psi_lo, float psi_hi, float frac, int k,
                              float *psi_out, int64_t *idx_out, int32_t *searched_out,
                              int out_flags);

/* Batched triaged search over the events of tcw_load_events against the
 * context's bank: the coarse pass of every event (patches of patch_size
 * Doppler-sorted skies of that event; patch_size = 0: ceil(n_sky / 32)
 * skies, i.e. 32 patches per event), ONE network call over all events'
 * patches, per event the ceil(frac * n_patch) best patches (spread apart by
 * TCW_OPT_TRIAGE_SPREAD), and one persistent group-kernel launch per wave over
 * the chosen (event, sky chunk, template group) items.  With
 * TCW_OPT_TRIAGE_TEMPLATES < 1000 each chosen patch contributes its
 * max(ceil(n_tmpl * permille / 1000), k) best templates by coarse Psi and an
 * event's chosen skies are searched over the union of its patches' templates;
 * otherwise over the whole bank, so that a searched row equals the row of
 * tcw_search_batched.  psi_out/idx_out [total_sky][k] as tcw_search_batched
 * for searched skies; rows of skipped skies hold -inf and -1.
 * searched_out [total_sky] (may be NULL): 1 for searched skies.  wbf and
 * theta are device pointers.  Runs eagerly (the selection changes with the
 * data, so it is not recorded as a graph); tcw_get_triage_info reports its
 * totals over the batch.
 * Errors: as tcw_search_batched and tcw_triage_features, INVALID_ARGUMENT
 * (frac not in (0, 1], patch_size < 0). */
tcw_status tcw_search_batched_triaged(tcw_ctx *ctx, const uint16_t *wbf, const float *theta,
                                      int patch_size, float psi_lo, float psi_hi, float frac, int k,
                                      float *psi_out, int64_t *idx_out, int32_t *searched_out,
                                      int out_flags);

/* Ranking of the triage (the first step of tcw_search_triaged, returned to
 * the caller): the coarse pass as tcw_triage_features, the network's score
 * (logit y of the MLP above) of every patch, and the patches by (score desc,
 * patch index asc).  score_out [n_patch] float32 and patch_order_out
 * [n_patch] int32 (patch indices) may be NULL; sky_order_out [n_sky] int32
 * (may be NULL) lists the caller sky indices patch by patch in that order,
 * each patch's skies in the search's Doppler-sorted order, so its first
 * skies are those a triaged search with frac = m / n_patch and
 * TCW_OPT_TRIAGE_SPREAD = 0 searches.  A caller can drive its own
 * follow-up from it (another frac, another search of the best skies)
 * without repeating the coarse pass.  wbf and theta are device pointers;
 * outputs are host or device memory by out_flags.  Errors: as
 * tcw_triage_features; INVALID_ARGUMENT (null weights). */
tcw_status tcw_triage_rank(tcw_ctx *ctx, const uint16_t *wbf, const float *theta, int patch_size,
                           float psi_lo, float psi_hi, float *score_out, int32_t *patch_order_out,
                           int32_t *sky_order_out, int out_flags);

typedef struct {
    int n_patch;
    int n_selected;             /* patches searched exhaustively */
    int64_t skies_searched;
    int64_t lookups_full;       /* sums of the exhaustive search of every sky */
    int64_t lookups_coarse;     /* sums of the coarse pass */
    int64_t lookups_searched;   /* sums of the exhaustive search of the selected skies */
    float coarse_ms, mlp_ms, search_ms;  /* device times */
    int64_t templates_searched; /* templates of the exhaustive part (TCW_OPT_TRIAGE_TEMPLATES) */
    int coarse_kernel;          /* coarse pass of the last call: 1 = the sweep form (one thread
                                   per template over every segment; used when the track series
                                   meet its error bounds and n_patch <= 128), 0 = one thread per
                                   (template, patch) */
    int coarse_parts;           /* sweep form: segment ranges per template (chosen to fill the
                                   device's resident blocks), 0 otherwise */
} tcw_triage_info;

tcw_status tcw_get_triage_info(tcw_ctx *ctx, tcw_triage_info *info);

/* The search's Doppler-sorted sky order: order_out[i] = caller index of the
 * i-th sky (host memory, n_sky entries).  Errors: STATE, INVALID_ARGUMENT. */
tcw_status tcw_sky_order(tcw_ctx *ctx, int32_t *order_out);

/* Measurement helper (not part of the method): best-of-`reps` read
 * bandwidth in GB/s of a kernel streaming 16-byte L2-cached loads over a
 * `bytes` device buffer `passes` times per launch, on the current device.
 * A buffer that fits in L2 (e.g. 64 MiB) measures L2, a larger one DRAM.
 * Errors: INVALID_ARGUMENT (bytes outside [1 MiB, 64 GiB], passes or reps
 * < 1, NULL), CUDA. */
tcw_status tcw_probe_read_bandwidth(int64_t bytes, int passes, int reps, double *gbps_out);

/* Measurement helper (not part of the method): best-of-`reps` rate in TFLOP/s
 * (2 flops per fused multiply-add) of a kernel running 8 independent fma
 * chains of `iters` steps per thread, 8 x 256 threads per SM, in double
 * (fp64 != 0) or float, on the current device.  Errors: INVALID_ARGUMENT
 * (iters or reps < 1, NULL), CUDA. */
tcw_status tcw_probe_fma_rate(int fp64, int iters, int reps, double *tflops_out);

/* Information about the last search. */
/* ---------------------------------------------------------------------------
 * Template banks generated on the device (Sec. 2 of arXiv:2507.07816 uses a
 * cubic lattice with equal spacing per axis and a uniform random bank over
 * (f0, tau, n)).  A bank is a pure function of its spec and the template
 * index t, so any range of a bank of 1e8-1e9 templates is produced alone:
 *   TCW_BANK_LATTICE  n_f0 x n_tau x n_n points, f0 fastest:
 *                     t -> (t mod n_f0, (t / n_f0) mod n_tau, t / (n_f0 n_tau));
 *                     the i-th of m points is lo (i = 0 or m = 1), hi
 *                     (i = m - 1), else fma(hi - lo, i / (m - 1), lo)
 *   TCW_BANK_RANDOM   n_tmpl templates; template t takes the 4 x 64-bit block
 *                     of Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011)
 *                     at counter (t, 0, 0, 0) and key (seed, 0); its first
 *                     three words x give u = (x >> 11) 2^-53 in [0, 1) and
 *                     f0, tau, n = fma(hi - lo, u, lo)
 * Bounds: finite, lo <= hi, f0_lo > 0, tau_lo > 0, n_lo > 1.
 * ------------------------------------------------------------------------- */
enum { TCW_BANK_LATTICE = 0, TCW_BANK_RANDOM = 1 };
typedef struct {
    int kind;                          /* TCW_BANK_LATTICE or TCW_BANK_RANDOM */
    int reserved;                      /* 0 */
    int64_t n_f0, n_tau, n_n;          /* lattice points per axis, each >= 1 */
    int64_t n_tmpl;                    /* random: number of templates >= 1 */
    double f0_lo, f0_hi;               /* Hz */
    double tau_lo, tau_hi;             /* s */
    double n_lo, n_hi;                 /* braking index */
    uint64_t seed;                     /* random: Philox key word 0 */
} tcw_bank_spec;

/* Number of templates of a spec (n_f0 n_tau n_n, or n_tmpl; at most 2^62).
 * Errors: INVALID_ARGUMENT (bad spec). */
tcw_status tcw_bank_size(const tcw_bank_spec *spec, int64_t *n_out);

/* Templates [first, first + count) of the bank, generated on the device, into
 * f0, tau, n (float64, count entries each; out_flags TCW_HOST or TCW_DEVICE).
 * Errors: INVALID_ARGUMENT (bad spec or range), OUT_OF_MEMORY, CUDA. */
tcw_status tcw_generate_bank(tcw_ctx *ctx, const tcw_bank_spec *spec, int64_t first, int64_t count,
                             double *f0, double *tau, double *n, int out_flags);

/* The templates of the bank at the indices idx[0 .. count) (host int64, each
 * in [0, bank size)), e.g. the idx_out of tcw_search_generated, into f0, tau,
 * n (float64, count entries; out_flags TCW_HOST or TCW_DEVICE).
 * Errors: INVALID_ARGUMENT (bad spec, index outside the bank), OUT_OF_MEMORY,
 * CUDA. */
tcw_status tcw_generate_bank_at(tcw_ctx *ctx, const tcw_bank_spec *spec, const int64_t *idx, int64_t count,
                                double *f0, double *tau, double *n, int out_flags);

/* Search a generated bank with the loaded spectrogram, velocities and sky,
 * like tcw_search: psi_out/idx_out [n_sky][k] with idx the generated template
 * index t (int64).  The bank is produced chunk by chunk on the device
 * (TCW_OPT_GEN_CHUNK templates), each chunk searched and its per-sky top-k
 * merged into a running top-k by (Psi desc, t asc), so the full Psi array is
 * never held: memory is one chunk's Psi (n_sky x chunk floats), whatever the
 * bank size.  Honours the statistic, amplitude, lanes and kernel options.
 * Replaces any bank defined with tcw_define_bank (define it again before
 * tcw_search); tcw_get_statistics is not available afterwards.
 * 1 <= k <= min(bank size, 1024).  Errors: as tcw_search, plus
 * INVALID_ARGUMENT for a bad spec. */
tcw_status tcw_search_generated(tcw_ctx *ctx, const tcw_bank_spec *spec, double T0, int k,
                                float *psi_out, int64_t *idx_out, int out_flags);

typedef struct {
    int64_t n_tmpl;             /* templates searched */
    int64_t chunks;             /* chunks (kernel passes over the data) */
    int64_t chunk_templates;    /* templates per chunk */
    int64_t lookups;            /* n_sky * n_tmpl * n_det * n_seg */
    int kernel;                 /* TCW_KERNEL_GROUP or TCW_KERNEL_LOOKUP (last chunk) */
    int launches;               /* kernels launched */
    float search_ms;            /* device time of the search kernels, summed over chunks */
    float total_ms;             /* device time from the first generation to the last merge */
} tcw_generated_info;

/* Information about the last tcw_search_generated.  Errors: STATE. */
tcw_status tcw_get_generated_info(tcw_ctx *ctx, tcw_generated_info *info);

typedef struct {
    int kernel;                 /* TCW_KERNEL_GROUP or TCW_KERNEL_LOOKUP */
    int launches;               /* kernels launched by the search */
    int64_t lookups;            /* n_sky * n_tmpl * n_det * n_seg */
    int64_t general_path_lanes; /* group-kernel (template, detector, segment,
                                   sky-group) steps that took the per-sky path */
    double doppler_bins_max;    /* largest |f * v.nhat/c| / df over the search */
    double quantum;             /* fixed-point step of the Doppler factor */
    float search_ms;            /* device time of the search kernel, ms */
} tcw_info;

tcw_status tcw_get_info(tcw_ctx *ctx, tcw_info *info);

const char *tcw_status_string(tcw_status status);
const char *tcw_last_error(tcw_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TCW_H */
