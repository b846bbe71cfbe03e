/*
 * vbmc.h -- C ABI of the GB300 verifier for MLPs over a discretised input
 * perturbation box (arXiv 1907.12933, "Incremental Bounded Model Checking of
 * Artificial Neural Networks in CUDA").
 *
 * The paper checks two things about a network given by its weights and
 * biases (Sec. III-C, checkNN; Sec. III-B, covering methods):
 *   - safety: every image in a region around a given image keeps the class
 *     of that image (Eq. 9 restricts the region, Eq. 10 states the property;
 *     a violation yields a counterexample image);
 *   - coverage: which neurons change sign (sign(u) = 1 iff u >= 0, sc) and
 *     which neuron pairs are SS-covered (Sec. III-B), and the covered
 *     fraction of Eq. 3.
 * This library decides both exactly over a finite region that replaces the
 * Euclidean ball of Eq. 9: s chosen pixels, each moved by an integer number
 * of grey levels in [-k, k] and clipped to [0, 255]. Point index t in
 * [0, R^s), R = 2k+1, is read as s base-R digits with the first listed pixel
 * most significant; digit d is the step d - k.
 *
 * Network semantics: activation potential u = sum_j w_j i_j + b (Eq. 1);
 * hidden layers apply sigmoid (Eq. 2), ReLU or identity; the output layer is
 * linear and the class is its argmax (lowest index on exact ties). A point
 * is adversarial iff its class differs from the class D of the unperturbed
 * image. Margin m = y_D - max_{i != D} y_i. Results agree with an FP64
 * evaluation of every point: a point with |m| < 1e-9 is a tie (listed, not
 * counted); a neuron evaluation with |u| < 1e-9 is a sign tie (its
 * contributions go to the tie masks).
 *
 * Conventions for every call:
 *   - Return value: VBMC_OK or a negative vbmc_status; no call aborts the
 *     process. vbmc_last_error() gives a message for the calling thread.
 *   - Ownership: the caller owns every input and may free it when the call
 *     returns. Handles (vbmc_net, vbmc_result) are owned by the library
 *     until the matching *_free. get_* calls copy into caller buffers.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     All device work of a call is ordered on it.
 *   - Memory: device memory is allocated by vbmc_net_create,
 *     vbmc_net_prepare, vbmc_result_create(_batch), vbmc_autotune, the proposal
 *     calls and the diagnostic vbmc_wide_trace. A verify call allocates
 *     nothing, except that the first call at a tensor precision on a net that
 *     was not prepared for it builds that precision's weight copies.
 *   - Errors found on the device (an invalid pixel list passed by device
 *     pointer, a full recheck queue) are latched in the result and returned
 *     by the next call that reads it.
 */
#ifndef VBMC_H
#define VBMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VBMC_MAX_LAYERS 8   /* weight layers                     */
#define VBMC_MAX_S 16       /* perturbed pixels per query        */
#define VBMC_MAX_K 127      /* steps per pixel (R = 2k+1 <= 255) */
#define VBMC_MAX_WIDTH 1024 /* neurons per layer                 */
#define VBMC_NO_WITNESS UINT64_MAX

typedef enum {
    VBMC_OK = 0,
    VBMC_ERR_ARG = -1,         /* invalid argument or buffer too small    */
    VBMC_ERR_OOM = -2,         /* device allocation or queue capacity     */
    VBMC_ERR_CUDA = -3,        /* CUDA runtime error                      */
    VBMC_ERR_TIMEOUT = -4,     /* time budget exhausted                   */
    VBMC_ERR_UNSUPPORTED = -5, /* shape or precision not supported        */
    VBMC_ERR_STATE = -6,       /* handle used in the wrong state          */
    VBMC_ERR_DEVICE = -7       /* error reported by a device-side check   */
} vbmc_status;

typedef enum { VBMC_ACT_IDENTITY = 0, VBMC_ACT_SIGMOID = 1, VBMC_ACT_RELU = 2 } vbmc_act;

/* Precision of the first pass over all points. Every pass except FP64
 * screens with a proven error bound; points it cannot decide are re-run in
 * a tighter precision and finally in FP64, so the results do not depend on
 * this choice. */
typedef enum {
    VBMC_PREC_FP64 = 0, /* every point in FP64 on CUDA cores              */
    VBMC_PREC_FP32 = 1, /* FP32 screen on CUDA cores (the plain GPU path) */
    VBMC_PREC_BF16 = 2, /* BF16 tcgen05 screen for layers 2..L            */
    VBMC_PREC_FP16 = 3, /* FP16 tcgen05 screen for layers 2..L            */
    VBMC_PREC_FP8 = 4   /* E4M3 tcgen05 screen, per-channel scales        */
} vbmc_precision;

typedef enum {
    VBMC_SAFE = 0,      /* no adversarial point, no tie                */
    VBMC_UNSAFE = 1,    /* at least one adversarial point              */
    VBMC_TIES_ONLY = 2, /* no adversarial point, some |m| < 1e-9 ties  */
    VBMC_PARTIAL = 3    /* the checked range is not the whole space    */
} vbmc_verdict;

/* Network: L weight layers, sizes H_0..H_L. W[l] is row-major
 * H_{l+1} x H_l (row i = weights of neuron i of layer l+1), b[l] has H_{l+1}
 * entries; host pointers, copied by vbmc_net_create. */
typedef struct {
    int32_t n_layers;
    const int32_t *dims;
    const float *const *W;
    const float *const *b;
    int32_t hidden_act; /* vbmc_act */
} vbmc_mlp_desc;

/* Query: base image (H_0 grey levels), s distinct pixel indices in digit
 * order, step bound k, and the index range [lo, hi) to check (hi = 0: the
 * whole space). Host pointers.
 * filter (0: every point of the box) restricts the checked points:
 *   VBMC_FILTER_L2     the perturbed image lies in the Euclidean ball of
 *                      Eq. 9 on the grid: sum over the s pixels of the clipped
 *                      change in grey levels squared <= l2_max (for a radius b
 *                      on the [0, 1] scale, l2_max = floor((255 b)^2))
 *   VBMC_FILTER_SHELL  the point lies on the box's boundary: some pixel is
 *                      moved by exactly k steps (one shell of the k-shell order)
 * Filtered-out points are not checked or counted (n_points counts the rest).
 * property selects what makes a point a counterexample:
 *   VBMC_PROP_ARGMAX     Eq. 10: argmax of the outputs differs from the
 *                        unperturbed image's class D (margin y_D - max_{i!=D}
 *                        y_i < 0); tie when |margin| < 1e-9
 *   VBMC_PROP_THRESHOLD  Eq. 11 with the reference value V = threshold:
 *                        y_D < V and y_i > V for some i != D, i.e. the margin
 *                        max(y_D - V, V - max_{i!=D} y_i) < 0; tie when
 *                        |margin| < 1e-9. threshold must be finite. */
enum { VBMC_FILTER_L2 = 1, VBMC_FILTER_SHELL = 2 };
enum { VBMC_PROP_ARGMAX = 0, VBMC_PROP_THRESHOLD = 1 };

typedef struct {
    const uint8_t *image;
    int32_t s;
    const int32_t *pixels;
    int32_t k;
    uint64_t lo, hi;
    int32_t filter;
    int64_t l2_max;
    int32_t property;  /* vbmc property enum above */
    double threshold;  /* VBMC_PROP_THRESHOLD: the reference value V */
} vbmc_query;

enum { VBMC_SCHED_GIVEN = 0, VBMC_SCHED_SMALL_FIRST = 1 };

typedef struct {
    int32_t precision;  /* vbmc_precision                                  */
    int32_t coverage;   /* nonzero: compute sign-change and SS masks       */
    int32_t bitmap;     /* nonzero: record the per-point verdict bitmap    */
    int32_t graph;      /* batch: nonzero captures the passes into one CUDA
                         * graph and launches it                          */
    int32_t schedule;   /* batch: VBMC_SCHED_GIVEN checks all queries' tiles
                         * in the given order, then their rechecks.
                         * VBMC_SCHED_SMALL_FIRST sorts the queries by point
                         * count (shortest job first) and runs them in up to
                         * 8 waves of about equal work, each a full chain of
                         * passes: a query is final when its wave ends   */
    double time_budget_ms; /* one query (verify_query / _device), BF16/FP16
                         * fused screen or FP32 path: device-time budget from
                         * the call's prologue, 0 for none. The first pass
                         * takes its tiles of [lo, hi) in index order and
                         * takes none after the budget; every tile taken is
                         * finished, rechecks included, so the result is exact
                         * for the checked prefix [lo, checked_hi) of the
                         * summary, and the call returns VBMC_ERR_TIMEOUT when
                         * that prefix is shorter than [lo, hi); the result
                         * handle then holds that prefix's result (summary and
                         * get_* calls read it). A timed-out check resumes
                         * with lo = checked_hi (results of ranges merge:
                         * sums, min, bitwise or). Other paths
                         * (FP64, FP8, wide layers, small nets, batches)
                         * check the whole range.                         */
} vbmc_options;

/* Capacities fixed when a result handle is created. */
typedef struct {
    uint64_t max_points; /* verdict bitmap bits (0: no bitmap)             */
    int32_t max_s;       /* <= VBMC_MAX_S                                  */
    int32_t max_k;       /* <= VBMC_MAX_K                                  */
    uint32_t ties_cap;   /* tie indices kept (all are counted)             */
    uint64_t queue_cap;  /* points that may wait for a tighter recheck     */
    int64_t wide_chunk;  /* nets with the wide-layer tensor path (ReLU,
                          * hidden widths a multiple of 256 up to 1024):
                          * points per chunk of its workspace, allocated
                          * here (about 4 x widest hidden layer + 250
                          * bytes per point). 0: min(2^20, (2 max_k + 1)
                          * ^ max_s); -1: none, and FP8 or wide BF16/FP16
                          * verify calls on this result fail with
                          * VBMC_ERR_STATE. Rounded up to 128.          */
} vbmc_caps;

typedef struct {
    int32_t verdict;           /* vbmc_verdict                            */
    int32_t D;                 /* class of the unperturbed image          */
    double base_margin;        /* FP64 margin of the unperturbed image    */
    uint64_t n_points;         /* points checked                          */
    uint64_t n_adversarial;    /* adversarial points (ties excluded)      */
    uint64_t first_witness;    /* smallest adversarial index, or NO_WITNESS */
    uint64_t n_ties;           /* points with |m| < 1e-9                  */
    uint64_t n_recheck[4];     /* points re-run: tensor split, FP32,      *
                                * double-float, FP64                      */
    double ms_device;          /* device time of the last verify call     */
    double ms_prologue;        /* of which: FP64 base pass and tables     */
    double ms_screen;          /* of which: first pass over every point   */
    double ms_recheck;         /* of which: all later passes              */
    double ms_to_verdict;      /* device time from the query's prologue to
                                * its final result (batch: per query)     */
    double ms_pass[4];         /* of the recheck time: split tensor pass,
                                * FP32 pass, double-float pass, FP64 pass
                                * (batch: first wave; wide-layer path: all
                                * in ms_screen, its chunks interleave)     */
    uint64_t checked_hi;       /* end of the checked prefix [lo, checked_hi)
                                * (hi unless the time budget ran out)      */
} vbmc_summary;

typedef struct vbmc_net vbmc_net;
typedef struct vbmc_result vbmc_result;

/* Copy a network, given only by its weights and biases as in checkNN's
 * first input (Sec. III-C), to the device. Computes the weight norms the
 * screens' error bounds use. Allocates device memory; not for the timed path. */
vbmc_status vbmc_net_create(const vbmc_mlp_desc *desc, vbmc_net **out);

/* Build the net's operands for a tensor precision now (BF16/FP16: the fused
 * screen's or the wide-layer path's rounded weights, their norms, and the
 * accumulator self-test; FP8: the E4M3 weights, scales and self-test), so that
 * no later verify call allocates. FP32 and FP64 need nothing (VBMC_OK).
 * VBMC_ERR_UNSUPPORTED when the net has no tensor path at that precision. */
vbmc_status vbmc_net_prepare(vbmc_net *net, int32_t precision);
vbmc_status vbmc_net_free(vbmc_net *net);

/* Allocate a reusable result workspace for queries on `net` within `caps`. */
vbmc_status vbmc_result_create(const vbmc_net *net, const vbmc_caps *caps, vbmc_result **out);

/* Allocate nq result workspaces that vbmc_verify_batch can serve with one
 * launch per pass: out[i] must then be passed as results[i]. caps.queue_cap
 * sizes the recheck queues the batch shares. Each handle is freed with
 * vbmc_result_free. */
vbmc_status vbmc_result_create_batch(const vbmc_net *net, const vbmc_caps *caps, int32_t nq,
                                     vbmc_result **out);
vbmc_status vbmc_result_free(vbmc_result *res);

/* checkNN over the box (Sec. III-C): enumerate [lo, hi), decide the safety
 * property of Eq. 10 for every point, collect the sign-change and SS-Cover
 * masks (Sec. III-B). Host inputs; blocks until the result is final. */
vbmc_status vbmc_verify_query(vbmc_net *net, const vbmc_query *query, const vbmc_options *opt,
                              vbmc_result *res, void *stream);

/* Same, with the image (H_0 bytes) and pixel list (s int32) already in
 * device memory. Asynchronous: enqueues the work on `stream` and returns;
 * the result stays on the device until a get_* call or vbmc_result_summary
 * reads it. Invalid pixel lists are detected on the device. */
vbmc_status vbmc_verify_query_device(vbmc_net *net, const uint8_t *d_image, int32_t s,
                                     const int32_t *d_pixels, int32_t k, uint64_t lo, uint64_t hi,
                                     const vbmc_options *opt, vbmc_result *res, void *stream);

/* checkNN (Sec. III-C) for many queries against one net: with results from one vbmc_result_create_batch
 * call (in order), every query's points go to one persistent launch per pass
 * (tiles never span queries; rechecked points of all queries share the
 * queues), optionally captured as one CUDA graph (opt->graph). Other result
 * handles are served one query after another. results[i] receives query i;
 * each summary's ms_to_verdict is that query's own time to a final result.
 * Blocks until all results are final. */
vbmc_status vbmc_verify_batch(vbmc_net *net, const vbmc_query *queries, int32_t nq,
                              const vbmc_options *opt, vbmc_result *const *results, void *stream);

/* Waits for the result's last call and returns its summary. */
vbmc_status vbmc_result_summary(vbmc_result *res, vbmc_summary *out);

/* First (lexicographically smallest) counterexample of the query's property
 * (Eq. 10, or Eq. 11): its index,
 * its s steps in [-k, k], the perturbed image (H_0 bytes) and its FP64
 * margin. Any output pointer may be NULL. With no witness, *index =
 * VBMC_NO_WITNESS and the other outputs are left untouched. */
vbmc_status vbmc_get_witness(vbmc_result *res, uint64_t *index, int32_t *steps, uint8_t *image,
                             double *margin_fp64);

/* Coverage masks (Sec. III-B). flip: one bit per non-input neuron, layers
 * 1..L back to back (bit n of word n/32). ss: one block per adjacent layer
 * pair (l, l+1), l = 1..L-1, bit j*H_{l+1} + i for pair (j in l, i in l+1).
 * *_tie: bits whose decision involved a sign tie. covered_fraction: Eq. 3,
 * neurons in at least one SS-covered pair over all non-input neurons. Any
 * pointer may be NULL; a non-NULL buffer shorter than needed is an error. */
vbmc_status vbmc_get_coverage(vbmc_result *res, uint32_t *flip, size_t flip_words,
                              uint32_t *flip_tie, uint32_t *ss, size_t ss_words, uint32_t *ss_tie,
                              double *covered_fraction);

/* Word counts of the coverage masks for a net. */
vbmc_status vbmc_mask_words(const vbmc_net *net, size_t *flip_words, size_t *ss_words);

/* Verdict bitmap: bit t set iff point t is adversarial (ties clear). */
vbmc_status vbmc_get_verdict_bitmap(vbmc_result *res, uint32_t *words, size_t n_words);

/* Tie indices (ascending) and their total count. */
vbmc_status vbmc_get_ties(vbmc_result *res, uint64_t *idx, size_t cap, uint64_t *n_ties);

/* Message for the last failing call of this thread. */
const char *vbmc_last_error(void);

/* ---- The covering methods over a set of input pairs (Sec. III-B; no
 * enumeration). For every pair (x1, x2) of H_0-byte images (grey levels), the
 * FP64 potentials of both inputs decide, per non-input neuron n and layer k:
 *   sc(n)  sign change (sign(u) = 1 iff u >= 0)
 *   vc(n)  value change: no sign change and max(|u1|, |u2|) >= g min(|u1|, |u2|)
 *   dc(k)  distance change: no neuron of layer k changes sign and the Euclidean
 *          distance of the layer's potential vectors is at least d
 * and the four covers are ORed over all pairs:
 *   SS (i, j)  i the only sign change of layer k, sc(j)   pair layout (as in
 *   SV (i, j)  i the only sign change of layer k, vc(j)    vbmc_get_coverage)
 *   DS (k, j)  dc(k) and sc(j)   layer layout: bit of neuron j (its index among
 *   DV (k, j)  dc(k) and vc(j)   the non-input neurons); covers (any i of k, j)
 * Undecided tests (|u| < 1e-9, |max - g min| <= 1e-9, |dist - d| <= 1e-9) go
 * to the tie masks as for SS. Every mask pointer is device memory of
 * vbmc_mask_words words (flip words for flip, DS, DV; SS words for SS, SV) or
 * NULL; masks are cleared by the call. Asynchronous on `stream`. */
typedef struct {
    double g; /* value-change ratio (>= 1)      */
    double d; /* distance-change bound (>= 0)   */
} vbmc_cover_params;

typedef struct {
    uint32_t *flip, *flip_tie;   /* sign changes                 */
    uint32_t *ss, *ss_tie;       /* SS-Cover, pair layout        */
    uint32_t *sv, *sv_tie;       /* SV-Cover, pair layout        */
    uint32_t *ds, *ds_tie;       /* DS-Cover, layer layout       */
    uint32_t *dv, *dv_tie;       /* DV-Cover, layer layout       */
} vbmc_pair_masks;

vbmc_status vbmc_pair_coverage(const vbmc_net *net, const uint8_t *d_images1, const uint8_t *d_images2,
                               int32_t n_pairs, const vbmc_cover_params *params,
                               const vbmc_pair_masks *out, void *stream);

/* The same covers over the enumeration: the pairs (x, x_t) of the query's
 * unperturbed image x and each point x_t of [lo, hi) (hi = 0: the whole box)
 * that passes the query's filter, in FP64 (x_t's layer 1 incrementally from
 * x's potentials, layers 2..L in full), with the definitions and tie masks of
 * vbmc_pair_coverage; flip and SS equal the masks of vbmc_verify_query for
 * the same points. The query's property is ignored. Uses res for staging (its
 * verify result is discarded). *n_points (may be NULL) receives the points
 * checked. Blocks until done. */
vbmc_status vbmc_enum_coverage(vbmc_net *net, const vbmc_query *query, const vbmc_cover_params *params,
                               const vbmc_pair_masks *out, vbmc_result *res, uint64_t *n_points,
                               void *stream);

/* Diagnostic of the wide-layer tensor path (FP8 E4M3, or BF16/FP16 on nets the
 * fused screen does not hold): verifies points [0, n_points) of the query at
 * that precision (coverage off) and returns, for each hidden layer l = 1..L-1
 * and point i, the layer's operand as the tensor cores consume it (the
 * rounded dh_l = h_l(point) - h_l(unperturbed), dequantized with the point's
 * scale) in vals[((l-1) n_points + i) H_max + j] (H_max = widest layer), and
 * in nre[((l-1) n_points + i) 3 + {0, 1, 2}] the path's N_l = ||dh_l||, R_l =
 * ||dh_l - operand|| and its proven bound E_l on ||dh_l - exact||, all rounded
 * up; so ||operand - exact dh_l|| <= R_l + E_l. Host output buffers. Allocates
 * and frees device scratch; n_points must not exceed the path's chunk of
 * points (2^20 by default). Blocks until done; res holds the verification. */
vbmc_status vbmc_wide_trace(vbmc_net *net, const vbmc_query *query, int32_t precision, int32_t n_points,
                            float *vals, float *nre, vbmc_result *res, void *stream);

/* Eq. 3-6: fraction of non-input neurons that belong to at least one covered
 * pair of a host mask in pair layout (SS, SV) or layer layout (DS, DV). */
enum { VBMC_LAYOUT_PAIRS = 0, VBMC_LAYOUT_LAYER = 1 };
vbmc_status vbmc_covered_fraction(const vbmc_net *net, int32_t layout, const uint32_t *mask,
                                  double *fraction);

/* ---- Launch-shape autotuning. The FP32 pass (over index ranges, and over
 * queued points) comes in six variants that hold layers up to 32, 256, 512,
 * 1024, 512 and 256 neurons with 128, 128, 64, 32, 32 and 64 points per
 * tile (variant numbers 1..6); it and the
 * double-float pass also take a number of CTAs per SM. vbmc_autotune times
 * every variant that fits the net, at 1, 2 and 4 CTAs per SM, and the
 * double-float pass at 2, 4, 8 and 16 CTAs per SM, on a sample box of the
 * net (s <= 4 pixels, R^s >= 2^17 points), keeps the fastest of each, and
 * applies them to the net. With cache_path set, a file of JSON lines keyed by
 * the net's shape, activation, SM count and compute capability is read first
 * (a hit skips the timing) and updated after a measurement. The choice never
 * changes results, only speed. Blocks until done; allocates a temporary
 * result workspace. */
typedef struct {
    int32_t simt_range, simt_range_ctas;   /* FP32 pass over ranges: variant, CTAs/SM */
    int32_t simt_gather, simt_gather_ctas; /* FP32 pass over queued points            */
    int32_t df_ctas;                       /* double-float pass CTAs/SM               */
    int32_t from_cache;                    /* 1: read from cache_path                 */
    double ms_range, ms_gather, ms_df;     /* best times measured (0 from the cache)  */
} vbmc_tuning;

vbmc_status vbmc_autotune(vbmc_net *net, const char *cache_path, vbmc_tuning *out);

/* Apply given launch shapes (0 in a field: the built-in choice). */
vbmc_status vbmc_set_tuning(vbmc_net *net, const vbmc_tuning *t);

/* Accumulation error per product that the FP8 screen's bound assumes for this
 * net's device, relative to the sum of |products|: 2^-22 when the set-up
 * self-test found the E4M3 MMA's sums exact to 23 significand bits (the FP32
 * model of the 16-bit screens), 2^-13 otherwise. Builds the FP8 weights on
 * first use. */
vbmc_status vbmc_fp8_accumulation_unit(vbmc_net *net, double *unit);

/* Accumulation error per product that the BF16 / FP16 screens' bounds use on
 * this device (precision VBMC_PREC_BF16 or VBMC_PREC_FP16), relative to the sum
 * of |products| of a dot product. The PTX ISA does not state how the kind::f16
 * MMA rounds its partial sums, so a set-up self-test measures it on the
 * screens' own operand layout (K = 256 over four chunks): integer tiles that
 * must come back exact (else VBMC_ERR_UNSUPPORTED), probe sums that need 17 to
 * 24 significand bits, and random operands checked against the model
 * K u sum |products|. *unit = 2^-22 (the FP32 model) when the probes are exact
 * and every output lies within the model at that unit, 2^-13 when only the
 * looser model holds. *worst (may be NULL) = the largest observed
 * |error| / (K sum |products|) over the test tile; *probes_failed (may be
 * NULL) = bit i set when probe i did not come back exact. Does not need the
 * net's weights; the result is kept per device and type. */
vbmc_status vbmc_tc_accumulation_unit(vbmc_net *net, int32_t precision, double *unit, double *worst,
                                      int32_t *probes_failed);

/* ---- k-shell order: the shells r = 0, 1, ..., k (points whose largest step
 * is exactly r, checked as the box of radius r restricted to its boundary)
 * one after another, stopping after the first shell that holds a point
 * violating Eq. 10; the smallest L-infinity witness comes first (the bound of
 * the incremental check grows until a counterexample or the bound k). The
 * query's own filter (VBMC_FILTER_L2) applies as well; lo and hi must be 0.
 * After the call the result holds the last shell checked (its summary, and
 * vbmc_get_witness with steps in [-radius, radius]). Without a witness every
 * shell was checked: the box is SAFE when n_ties is 0. Blocks until done. */
typedef struct {
    int32_t radius;           /* shell of the first witness, -1: none up to k */
    uint64_t points_checked;  /* over all shells checked                      */
    uint64_t n_ties;          /* margin ties over all shells checked          */
    double ms_device;         /* device time over all shells checked          */
} vbmc_shell_out;

vbmc_status vbmc_shell_search(vbmc_net *net, const vbmc_query *query, const vbmc_options *opt,
                              vbmc_result *res, vbmc_shell_out *out, void *stream);

/* ---- Tile-ordered search for a first witness.
 * The index space [0, n) of a query (n = R^s) is cut into n_tiles contiguous
 * tiles of ceil(n / n_tiles) points (the last one ragged; tiles past n are
 * empty). vbmc_search_query checks the tiles in the order given by `order`
 * (a permutation of 0..n_tiles-1, host memory) with the same exact pipeline
 * as vbmc_verify_query, and stops after the first tile that holds a point
 * violating Eq. 10. Without any witness every tile is checked, and the
 * verdict is the one vbmc_verify_query gives (SAFE or TIES_ONLY). After the
 * call, vbmc_result_summary reports the checked points (n_points), the
 * adversarial points found in the checked tiles, and the smallest of them
 * (first_witness, the first in index order within the witness tile); the
 * verdict is UNSAFE once a witness is found, PARTIAL is never reported.
 * Coverage masks and the verdict bitmap, when requested, cover the checked
 * tiles only. Blocks until the search ends. */
typedef struct {
    int32_t tiles_checked;      /* tiles checked, the witness tile included        */
    int32_t witness_tile;       /* tile holding the first witness found, or -1     */
    uint64_t points_checked;
    double ms_to_witness;       /* device time from the start of the query's set-up
                                   to the end of the witness tile (or of the last
                                   tile without a witness)                          */
} vbmc_search_out;

vbmc_status vbmc_search_query(vbmc_net *net, const vbmc_query *query, int32_t n_tiles,
                              const int32_t *order, const vbmc_options *opt, vbmc_result *res,
                              vbmc_search_out *out, void *stream);

/* Adversarial points per tile (n_tiles tiles as above, at most
 * VBMC_MAX_TILES) from the verdict bitmap of the result's last call, which must
 * have covered the whole space with the bitmap on. counts: n_tiles uint64 in
 * host memory; the device counters are the result's own (no allocation). */
#define VBMC_MAX_TILES 1024
vbmc_status vbmc_tile_counts(vbmc_result *res, int32_t n_tiles, uint64_t *counts);

/* ---- Learned tile proposal: a 3-layer MLP (F -> H1 -> H2 -> T, ReLU hidden
 * layers) trained on the GPU to rank the T tiles of a query so that
 * vbmc_search_query meets a witness sooner. Weights are FP32 masters; the
 * scoring forward and the training forward round weights and activations to
 * BF16 (FP32 accumulation). Not a part of the exact check: any order yields
 * the same verdicts. All pointers named d_* are device memory. */
typedef struct vbmc_proposal vbmc_proposal;

/* He-normal weights from `seed`, zero biases; max_batch bounds B below.
 * n_tiles in [2, 1024]. */
vbmc_status vbmc_proposal_create(int32_t n_features, int32_t h1, int32_t h2, int32_t n_tiles,
                                 int32_t max_batch, uint64_t seed, vbmc_proposal **out);
vbmc_status vbmc_proposal_free(vbmc_proposal *p);

/* Features of nq queries on a ReLU net, 3 * H_0 floats per query (row-major
 * [nq][3 * H_0]): the image / 255; at the p-th listed pixel the place value
 * R^-p of its digit, 0 elsewhere; and that place value times the input
 * gradient of the margin y_D - y_r (runner-up r) at the unperturbed image,
 * times k / 255, over the margin, clipped to [-16, 16]. d_images: [nq][H_0]
 * bytes; d_pixels: [nq][pix_stride] int32 (the first s[q] used); d_s, d_k:
 * [nq] int32. d_reach[q] (optional): sum over the listed pixels of
 * |gradient| * k / 255 over the margin (the first-order reach of the box);
 * d_margin[q] (optional): the FP32 margin. Asynchronous on `stream`. */
vbmc_status vbmc_proposal_features(const vbmc_net *net, const uint8_t *d_images,
                                   const int32_t *d_pixels, const int32_t *d_s, const int32_t *d_k,
                                   int32_t pix_stride, int32_t nq, float *d_features,
                                   float *d_reach, float *d_margin, void *stream);

/* Tile scores [B][T] of B feature rows [B][F]; with d_order non-NULL also
 * each row's tile order [B][T] (descending score, lower tile first on equal
 * scores). Asynchronous on `stream`. */
vbmc_status vbmc_proposal_scores(vbmc_proposal *p, const float *d_X, int32_t B, float *d_scores,
                                 int32_t *d_order, void *stream);

/* Loss and gradients of a batch: d_T [B][T] holds 0/1 witness labels per tile;
 * loss = mean over rows with a witness tile of -sum_i (t_i / sum t) log
 * softmax(z)_i. bf16 = 0 runs the forward in FP32 (for gradient checks).
 * *h_loss (optional) receives the loss; the call then waits for the stream.
 * Gradients are read with vbmc_proposal_params. */
vbmc_status vbmc_proposal_grads(vbmc_proposal *p, const float *d_X, const float *d_T, int32_t B,
                                int32_t bf16, float *h_loss, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with decoupled weight decay on
 * the weights, from the gradients of a BF16-forward batch. */
vbmc_status vbmc_proposal_train_step(vbmc_proposal *p, const float *d_X, const float *d_T, int32_t B,
                                     float lr, float weight_decay, float *h_loss, void *stream);

/* Copy layer l (1..3) weights [H_l][H_{l-1}], biases and last gradients to
 * host buffers (any may be NULL), or set the weights and biases. Synchronous. */
vbmc_status vbmc_proposal_params(vbmc_proposal *p, int32_t layer, float *h_W, float *h_b,
                                 float *h_gW, float *h_gb);
vbmc_status vbmc_proposal_set_params(vbmc_proposal *p, int32_t layer, const float *h_W,
                                     const float *h_b);

/* ---- For callers that cannot allocate device memory (no counterpart in the
 * paper). A process embedded in another runtime's memory pool, or one whose
 * allocator must not be re-entered, cannot call cudaMalloc. This entry point
 * runs the exhaustive FP64 check of [lo, hi) (the same results as
 * vbmc_verify_query with VBMC_PREC_FP64) and allocates nothing: all of its
 * per-query scratch sits in one fixed device array inside the library, and
 * the results go only into the caller's device buffers below.
 *   - Limits: at most VBMC_NOALLOC_MAX_NEURONS non-input neurons and
 *     s * (2k + 1) <= VBMC_NOALLOC_MAX_SR; larger queries get
 *     VBMC_ERR_UNSUPPORTED.
 *   - The array (128 KB) stays on every GPU that loads the library until the
 *     process exits. The first call on a device looks up its address; make
 *     that first call before capturing any stream into a graph.
 *   - Every call shares the array: calls whose GPU work overlaps (different
 *     streams, threads or processes sharing a context) race. Serialise them.
 *   - The caller's buffers are cleared by each call. The net must come from
 *     vbmc_net_create (done earlier, where allocation is allowed).
 * Asynchronous on `stream`; the outputs are valid once the stream reaches the
 * call's end. */
#define VBMC_NOALLOC_MAX_NEURONS 4096
#define VBMC_NOALLOC_MAX_SR 4096
#define VBMC_NOALLOC_BAD_PIXELS 1u /* flags in the high word of counters[3] */
#define VBMC_NOALLOC_TIES_CUT 4u

typedef struct {
    uint64_t *counters;      /* [4]: adversarial count, first witness (UINT64_MAX: none),
                                tie count, and class D of the unperturbed image in the
                                low 32 bits with flags in the high 32 bits:
                                VBMC_NOALLOC_BAD_PIXELS  the pixel list was invalid (not
                                                         distinct or out of range): no
                                                         other output is meaningful
                                VBMC_NOALLOC_TIES_CUT    more ties than ties_cap (or
                                                         ties == NULL): the count is
                                                         exact, the list holds the first
                                                         ties_cap found               */
    uint32_t *flip, *flip_tie, *ss, *ss_tie; /* coverage masks: all four, or all NULL   */
    uint32_t *bitmap;        /* verdict bits (bit t), or NULL                           */
    uint64_t bitmap_bits;    /* capacity of `bitmap` in bits                            */
    uint64_t *ties;          /* tie indices, unordered, or NULL                         */
    uint32_t ties_cap;
} vbmc_noalloc_out;

vbmc_status vbmc_verify_range_fp64_noalloc(const vbmc_net *net, const uint8_t *d_image, int32_t s,
                                           const int32_t *d_pixels, int32_t k, uint64_t lo,
                                           uint64_t hi, const vbmc_noalloc_out *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VBMC_H */
