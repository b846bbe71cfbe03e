/*
 * vbmc_oracle.c -- plain, slow FP64 CPU oracle for exhaustive verification of
 * an MLP over a discretised input-perturbation box.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file. It shares no code, header,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * What it computes, per point, from scratch and in double precision:
 *   - the neuron activation potential u = sum_j w_j * i_j + b        (Eq. 1)
 *   - the neuron output N(u) = 1 / (1 + e^-u) for sigmoid nets        (Eq. 2)
 *     or max(0, u) for ReLU nets (Sec. II-A lists ReLU as common); the
 *     output layer is left linear, so the class is the argmax of u_L
 *   - the safety property: the perturbed image must keep the class D of the
 *     unperturbed image (Eq. 10); a point is adversarial iff the argmax of
 *     its output differs from D, lowest index winning exact ties; or, on
 *     request, the misclassified literal of Eq. 11 with a reference value V:
 *     a point is adversarial iff y_D < V and y_i > V for some i != D
 *   - sign(u) = 1 if u >= 0 else 0, and the sign change sc between the
 *     unperturbed and the perturbed image for every non-input neuron
 *     (Sec. III-B, covering methods)
 *   - SS-Cover: pair (j in layer l, i in layer l+1) is covered iff j is the
 *     only neuron of layer l whose sign changed and i's sign changed
 *     (Sec. III-B, worked through in the Table I discussion and Table II)
 *   - the covered fraction of Eq. 3 over all non-input neurons.
 *
 * The perturbation space replaces the Euclidean ball of Eq. 9 with a box:
 * s chosen pixels, each shifted by an integer step in [-k, k] (units of
 * 1/255) and clipped to [0, 255]. Point index t is read as s digits of radix
 * R = 2k+1 with the first listed pixel as the most significant digit; digit
 * d means step d - k.
 *
 * Ties: a margin with |m| < 1e-9 is a tie (listed, not counted, its verdict
 * bit left clear); under Eq. 11, a verdict that rests on a comparison
 * |y - V| < 1e-9 is a tie. A neuron evaluation with |u| < 1e-9 (or whose unperturbed
 * value has |u| < 1e-9) is a sign tie: its flip goes to the tie mask, and any
 * SS pair whose decision depends on it goes to the SS tie mask.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ACT_IDENTITY 0
#define ORC_ACT_SIGMOID 1
#define ORC_ACT_RELU 2

typedef struct {
    int L;                   /* number of weight layers                      */
    const int *dims;         /* L+1 sizes H_0..H_L                           */
    const float *const *W;   /* W[l]: H_{l+1} x H_l, row i = neuron i        */
    const float *const *b;   /* b[l]: H_{l+1}                                */
    int act;                 /* hidden activation                            */
} orc_net;

typedef struct {
    /* inputs */
    const uint8_t *image;    /* H_0 grey levels                              */
    int s;
    const int *pixels;
    int k;
    uint64_t lo, hi;         /* hi == 0: whole space                         */
    double tau;              /* tie band, 1e-9                               */
    /* outputs (caller-owned; masks and bitmap must be zeroed by caller)     */
    uint32_t *bitmap;        /* bit t set iff t adversarial (non-tie)        */
    uint32_t *flip, *flip_tie, *ss, *ss_tie;
    uint64_t *ties;          /* tie indices, ascending, up to ties_cap       */
    uint64_t ties_cap;
    int D;
    double base_margin;
    uint64_t n_points, n_adv, first_witness, n_ties;
    /* input: which points of the box are checked (0: all). Bit 1: the perturbed
     * image within the Euclidean ball of Eq. 9 on the grid, sum over the pixels
     * of (clipped change in grey levels)^2 <= l2max. Bit 2: the point on the
     * box's boundary, some pixel moved by exactly k steps (a k-shell). Points
     * outside are neither checked nor counted. */
    int filter;
    long long l2max;
    /* input: 0 the property of Eq. 10 (argmax), 1 the misclassified literal of
     * Eq. 11 with reference value V */
    int property;
    double V;
} orc_query;

/* ---------------------------------------------------------------- basics */

static double orc_activation(int act, double u)
{
    if (act == ORC_ACT_SIGMOID) return 1.0 / (1.0 + exp(-u));   /* Eq. 2 */
    if (act == ORC_ACT_RELU) return u > 0.0 ? u : 0.0;
    return u;
}

static int orc_sign(double u) { return u >= 0.0 ? 1 : 0; }      /* sign(0) = 1 */

int orc_total_neurons(int L, const int *dims)
{
    int n = 0;
    for (int l = 1; l <= L; l++) n += dims[l];
    return n;
}

/* SS bits: one block per adjacent pair (layer l, layer l+1), l = 1..L-1,
 * bit (j -> i) at offset_l + j * H_{l+1} + i. */
uint64_t orc_ss_bits(int L, const int *dims)
{
    uint64_t n = 0;
    for (int l = 1; l < L; l++) n += (uint64_t)dims[l] * (uint64_t)dims[l + 1];
    return n;
}

/* Radix R = 2k+1, space size R^s; 0 if it does not fit below 2^63. */
uint64_t orc_space_size(int s, int k)
{
    uint64_t R = (uint64_t)(2 * k + 1), n = 1;
    for (int p = 0; p < s; p++) {
        if (n > (UINT64_C(1) << 62) / R) return 0;
        n *= R;
    }
    return n;
}

/* t -> digits, first pixel most significant. */
void orc_digits(uint64_t t, int s, int k, int *d)
{
    uint64_t R = (uint64_t)(2 * k + 1);
    for (int p = s - 1; p >= 0; p--) {
        d[p] = (int)(t % R);
        t /= R;
    }
}

/* Perturbed image of point t as doubles x = v'/255. */
void orc_point_image(const orc_net *net, const uint8_t *image, int s, const int *pixels,
                     int k, uint64_t t, double *x)
{
    int H0 = net->dims[0];
    int d[64];
    for (int j = 0; j < H0; j++) x[j] = (double)image[j] / 255.0;
    orc_digits(t, s, k, d);
    for (int p = 0; p < s; p++) {
        int v = (int)image[pixels[p]] + d[p] - k;
        if (v < 0) v = 0;
        if (v > 255) v = 255;
        x[pixels[p]] = (double)v / 255.0;
    }
}

/* Full forward pass. u_all receives the activation potentials of layers
 * 1..L back to back (Eq. 1); the hidden outputs use the activation, the
 * last layer stays linear. h0, h1: scratch of max(H) doubles each. */
void orc_forward(const orc_net *net, const double *x, double *u_all, double *h0, double *h1)
{
    const double *in = x;
    double *out = h0;
    int off = 0;
    for (int l = 0; l < net->L; l++) {
        int n_in = net->dims[l], n_out = net->dims[l + 1];
        const float *W = net->W[l];
        const float *b = net->b[l];
        for (int i = 0; i < n_out; i++) {
            double acc = 0.0;
            for (int j = 0; j < n_in; j++) acc += (double)W[(size_t)i * n_in + j] * in[j];
            double u = acc + (double)b[i];
            u_all[off + i] = u;
            out[i] = (l + 1 < net->L) ? orc_activation(net->act, u) : u;
        }
        off += n_out;
        in = out;
        out = (out == h0) ? h1 : h0;
    }
}

/* Class of an output vector: argmax, lowest index on exact ties. */
int orc_argmax(const double *y, int n)
{
    int best = 0;
    for (int i = 1; i < n; i++)
        if (y[i] > y[best]) best = i;
    return best;
}

/* Margin of class D: y_D - max_{i != D} y_i. */
double orc_margin(const double *y, int n, int D)
{
    double m = -INFINITY;
    for (int i = 0; i < n; i++)
        if (i != D && y[i] > m) m = y[i];
    return y[D] - m;
}

/* Eq. 11, the misclassified literal (n_D < V) and (n_i > V) for some i != D,
 * evaluated in three-valued logic: each comparison of an output with V is
 * undecided when |y - V| < tau. Returns 1 (true: the point is a
 * counterexample), 0 (false) or 2 (the truth value rests on an undecided
 * comparison: a tie). */
int orc_threshold_literal(const double *y, int n, int D, double V, double tau)
{
    int lit_d;   /* n_D < V */
    if (y[D] - V <= -tau) lit_d = 1;
    else if (y[D] - V >= tau) lit_d = 0;
    else lit_d = 2;
    int any = 0; /* some i != D with n_i > V */
    for (int i = 0; i < n; i++) {
        if (i == D) continue;
        if (y[i] - V >= tau) any = 1;
        else if (y[i] - V > -tau && any == 0) any = 2;
    }
    if (lit_d == 0 || any == 0) return 0;
    if (lit_d == 1 && any == 1) return 1;
    return 2;
}

/* A signed distance of Eq. 11 from holding: max(y_D - V, V - max_{i != D} y_i),
 * negative iff the literal holds. */
double orc_threshold_margin(const double *y, int n, int D, double V)
{
    double m = -INFINITY;
    for (int i = 0; i < n; i++)
        if (i != D && y[i] > m) m = y[i];
    double a = y[D] - V, b = V - m;
    return a > b ? a : b;
}

static void set_bit(uint32_t *w, uint64_t b) { w[b >> 5] |= 1u << (b & 31); }

/* Sign-change and SS-Cover contributions of one pair of inputs (x1, x2),
 * given their activation potentials u1, u2 over layers 1..L. */
static void orc_pair_coverage_scratch(int L, const int *dims, const double *u1,
                                      const double *u2, double tau, uint32_t *flip,
                                      uint32_t *flip_tie, uint32_t *ss, uint32_t *ss_tie,
                                      char *fl, char *ti)
{
    int total = orc_total_neurons(L, dims);
    /* fl: certain sign change; ti: sign tie */
    for (int n = 0; n < total; n++) {
        ti[n] = (fabs(u1[n]) < tau) || (fabs(u2[n]) < tau);
        fl[n] = (orc_sign(u1[n]) != orc_sign(u2[n])) && !ti[n];
        if (fl[n] && flip) set_bit(flip, (uint64_t)n);
        if (ti[n] && flip_tie) set_bit(flip_tie, (uint64_t)n);
    }
    int off = 0;
    uint64_t ss_off = 0;
    for (int l = 1; l < L; l++) {
        int Hl = dims[l], Hn = dims[l + 1];
        int n_flip = 0, n_tie = 0, only = -1;
        for (int j = 0; j < Hl; j++) {
            if (fl[off + j]) { n_flip++; only = j; }
            if (ti[off + j]) n_tie++;
        }
        for (int j = 0; j < Hl; j++) {
            /* j can be "the only changed neuron of layer l" for certain, or
             * only under some resolution of the ties. */
            int certain = (n_tie == 0 && n_flip == 1 && j == only);
            int possible = certain || (n_tie > 0 && ((n_flip == 1 && j == only) ||
                                                     (n_flip == 0 && ti[off + j])));
            if (!possible) continue;
            for (int i = 0; i < Hn; i++) {
                int ni = off + Hl + i;
                uint64_t bit = ss_off + (uint64_t)j * Hn + i;
                if (certain && fl[ni]) {
                    if (ss) set_bit(ss, bit);
                } else if (fl[ni] || ti[ni]) {
                    if (ss_tie) set_bit(ss_tie, bit);
                }
            }
        }
        off += Hl;
        ss_off += (uint64_t)Hl * Hn;
    }
}

void orc_pair_coverage(int L, const int *dims, const double *u1, const double *u2, double tau,
                       uint32_t *flip, uint32_t *flip_tie, uint32_t *ss, uint32_t *ss_tie)
{
    int total = orc_total_neurons(L, dims);
    char *fl = (char *)malloc((size_t)total);
    char *ti = (char *)malloc((size_t)total);
    orc_pair_coverage_scratch(L, dims, u1, u2, tau, flip, flip_tie, ss, ss_tie, fl, ti);
    free(fl);
    free(ti);
}

/* Eq. 3: fraction of non-input neurons that belong to at least one
 * SS-covered pair. */
double orc_ss_covered_fraction(int L, const int *dims, const uint32_t *ss)
{
    int total = orc_total_neurons(L, dims);
    char *cov = (char *)calloc((size_t)total, 1);
    int off = 0;
    uint64_t ss_off = 0;
    for (int l = 1; l < L; l++) {
        int Hl = dims[l], Hn = dims[l + 1];
        for (int j = 0; j < Hl; j++)
            for (int i = 0; i < Hn; i++) {
                uint64_t bit = ss_off + (uint64_t)j * Hn + i;
                if ((ss[bit >> 5] >> (bit & 31)) & 1u) {
                    cov[off + j] = 1;
                    cov[off + Hl + i] = 1;
                }
            }
        off += Hl;
        ss_off += (uint64_t)Hl * Hn;
    }
    int c = 0;
    for (int n = 0; n < total; n++) c += cov[n];
    free(cov);
    return (double)c / (double)total;
}

/* ---------------------------------------------------- the other covers */

/*
 * Sec. III-B, for one input pair (potentials u1, u2 of every non-input neuron):
 *   vc(n): the sign did not change and the value changed by the ratio g:
 *          max(|u1|, |u2|) >= g min(|u1|, |u2|)   (g > 1; the ratio is taken in
 *          whichever direction is >= 1)
 *   dc(k): no neuron of layer k changed sign and the Euclidean distance of the
 *          layer's potential vectors is at least d
 *   DS  pair (any i in layer k, j in layer k+1): dc(k) and sc(j)
 *   DV  pair (any i in layer k, j in layer k+1): dc(k) and vc(j)
 *   SV  pair (i in layer k, j in layer k+1): i is the only neuron of layer k
 *       that changed sign, and vc(j)
 * DS and DV are recorded per (layer k+1, neuron j): bit (offset of layer k+1 in
 * the non-input neurons) + j; SV uses the SS layout.
 * Ties, as for SS: a sign with |u| < tau in either input, a ratio test
 * |max - g min| <= tau, or a distance test |dist - d| <= tau is undecided; a
 * pair that holds only under some resolution of the undecided tests goes to
 * the tie mask, one that holds for every resolution to the mask itself.
 */
void orc_pair_covers(int L, const int *dims, const double *u1, const double *u2, double tau,
                     double g, double d, uint32_t *ds, uint32_t *ds_tie, uint32_t *dv,
                     uint32_t *dv_tie, uint32_t *sv, uint32_t *sv_tie)
{
    int total = orc_total_neurons(L, dims);
    char *fl = (char *)malloc((size_t)total);  /* certain sign change      */
    char *ti = (char *)malloc((size_t)total);  /* sign tie                 */
    char *vc = (char *)malloc((size_t)total);  /* certain value change     */
    char *vt = (char *)malloc((size_t)total);  /* value change undecided   */
    for (int n = 0; n < total; n++) {
        ti[n] = (fabs(u1[n]) < tau) || (fabs(u2[n]) < tau);
        fl[n] = (orc_sign(u1[n]) != orc_sign(u2[n])) && !ti[n];
        double a = fabs(u1[n]), b = fabs(u2[n]);
        double big = a > b ? a : b, small = a > b ? b : a;
        double test = big - g * small;
        vc[n] = !fl[n] && !ti[n] && test > tau;
        vt[n] = !fl[n] && !vc[n] && (ti[n] || fabs(test) <= tau);
    }
    int off = 0;
    uint64_t pair_off = 0;
    for (int l = 1; l < L; l++) {
        int Hl = dims[l], Hn = dims[l + 1];
        int n_flip = 0, n_tie = 0, only = -1;
        double dist2 = 0.0;
        for (int j = 0; j < Hl; j++) {
            if (fl[off + j]) { n_flip++; only = j; }
            if (ti[off + j]) n_tie++;
            double e = u1[off + j] - u2[off + j];
            dist2 += e * e;
        }
        double dist = sqrt(dist2);
        int dc_cert = n_flip == 0 && n_tie == 0 && dist - d > tau;
        int dc_poss = n_flip == 0 && dist - d >= -tau;
        for (int i = 0; i < Hn; i++) {
            int ni = off + Hl + i;
            uint64_t bit = (uint64_t)(off + Hl + i);
            /* DS */
            if (dc_cert && fl[ni]) { if (ds) set_bit(ds, bit); }
            else if (dc_poss && (fl[ni] || ti[ni])) { if (ds_tie) set_bit(ds_tie, bit); }
            /* DV */
            if (dc_cert && vc[ni]) { if (dv) set_bit(dv, bit); }
            else if (dc_poss && (vc[ni] || vt[ni])) { if (dv_tie) set_bit(dv_tie, bit); }
        }
        /* SV: the "only changed neuron" rule of SS with a value change above */
        for (int j = 0; j < Hl; j++) {
            int certain = (n_tie == 0 && n_flip == 1 && j == only);
            int possible = certain || (n_tie > 0 && ((n_flip == 1 && j == only) ||
                                                     (n_flip == 0 && ti[off + j])));
            if (!possible) continue;
            for (int i = 0; i < Hn; i++) {
                int ni = off + Hl + i;
                uint64_t bit = pair_off + (uint64_t)j * Hn + i;
                if (certain && vc[ni]) {
                    if (sv) set_bit(sv, bit);
                } else if (vc[ni] || vt[ni]) {
                    if (sv_tie) set_bit(sv_tie, bit);
                }
            }
        }
        off += Hl;
        pair_off += (uint64_t)Hl * Hn;
    }
    free(fl);
    free(ti);
    free(vc);
    free(vt);
}

/* Eq. 4 / Eq. 6: fraction of non-input neurons in at least one DS (DV) covered
 * pair; a bit of layer k+1 neuron j covers the pairs (i, j) for every i in layer k. */
double orc_layer_pair_fraction(int L, const int *dims, const uint32_t *mask)
{
    int total = orc_total_neurons(L, dims);
    char *cov = (char *)calloc((size_t)total, 1);
    int off = 0;
    for (int l = 1; l < L; l++) {
        int Hl = dims[l], Hn = dims[l + 1];
        for (int i = 0; i < Hn; i++) {
            uint64_t bit = (uint64_t)(off + Hl + i);
            if ((mask[bit >> 5] >> (bit & 31)) & 1u) {
                cov[off + Hl + i] = 1;
                for (int j = 0; j < Hl; j++) cov[off + j] = 1;
            }
        }
        off += Hl;
    }
    int c = 0;
    for (int n = 0; n < total; n++) c += cov[n];
    free(cov);
    return (double)c / (double)total;
}

/* ---------------------------------------------------------- enumeration */

typedef struct {
    const orc_net *net;
    const orc_query *q;
    const double *u_base;
    int D;
    uint64_t a, b;           /* this worker's range */
    size_t flip_words, ss_words;
    uint32_t *flip, *flip_tie, *ss, *ss_tie;
    uint64_t n_adv, first, n_ties, ties_len, ties_cap, n_points;
    uint64_t *ties;
    int status;
} orc_work;

static void *orc_worker(void *arg)
{
    orc_work *w = (orc_work *)arg;
    const orc_net *net = w->net;
    const orc_query *q = w->q;
    int H0 = net->dims[0], L = net->L, HL = net->dims[L];
    int hmax = 0;
    for (int l = 0; l <= L; l++) if (net->dims[l] > hmax) hmax = net->dims[l];
    int total = orc_total_neurons(L, net->dims);
    double *x = (double *)malloc(sizeof(double) * H0);
    double *u = (double *)malloc(sizeof(double) * total);
    double *h0 = (double *)malloc(sizeof(double) * hmax);
    double *h1 = (double *)malloc(sizeof(double) * hmax);
    char *fl = (char *)malloc((size_t)total);
    char *ti = (char *)malloc((size_t)total);
    w->first = UINT64_MAX;
    int R = 2 * q->k + 1;
    for (uint64_t t = w->a; t < w->b; t++) {
        if (q->filter) {
            /* digits of t, first pixel most significant; digit d is the step d - k */
            uint64_t tt = t;
            long long s2 = 0;
            int on_shell = q->k == 0;
            for (int p = q->s - 1; p >= 0; p--) {
                int d = (int)(tt % (uint64_t)R);
                tt /= (uint64_t)R;
                int v = q->image[q->pixels[p]];
                int vp = v + d - q->k;
                if (vp < 0) vp = 0;
                if (vp > 255) vp = 255;
                s2 += (long long)(vp - v) * (vp - v);
                if (d == 0 || d == R - 1) on_shell = 1;
            }
            if ((q->filter & 1) && s2 > q->l2max) continue;
            if ((q->filter & 2) && !on_shell) continue;
        }
        w->n_points++;
        orc_point_image(net, q->image, q->s, q->pixels, q->k, t, x);
        orc_forward(net, x, u, h0, h1);
        const double *y = u + (total - HL);
        int adv, tie;
        if (q->property == 1) {
            int lit = orc_threshold_literal(y, HL, w->D, q->V, q->tau);
            adv = lit == 1;
            tie = lit == 2;
        } else {
            adv = orc_argmax(y, HL) != w->D;
            tie = fabs(orc_margin(y, HL, w->D)) < q->tau;
        }
        if (tie) {
            if (w->ties_len == w->ties_cap) {
                w->ties_cap = w->ties_cap ? 2 * w->ties_cap : 64;
                w->ties = (uint64_t *)realloc(w->ties, sizeof(uint64_t) * w->ties_cap);
            }
            w->ties[w->ties_len++] = t;
            w->n_ties++;
        } else if (adv) {
            w->n_adv++;
            if (t < w->first) w->first = t;
            if (q->bitmap) set_bit(q->bitmap, t);  /* words are private to this worker */
        }
        if (w->flip)
            orc_pair_coverage_scratch(L, net->dims, w->u_base, u, q->tau, w->flip, w->flip_tie,
                                      w->ss, w->ss_tie, fl, ti);
    }
    free(x); free(u); free(h0); free(h1); free(fl); free(ti);
    return NULL;
}

/* Exhaustive check of [lo, hi). Returns 0 on success, -1 on bad arguments.
 * Coverage masks are computed when q->flip is non-NULL (then all four mask
 * pointers must be valid). */
int orc_verify(const orc_net *net, orc_query *q, int nthreads)
{
    int L = net->L, H0 = net->dims[0], HL = net->dims[L];
    if (L < 1 || HL < 2 || q->s < 0 || q->s > 64 || q->k < 0) return -1;
    if (q->property != 0 && (q->property != 1 || !isfinite(q->V))) return -1;
    for (int p = 0; p < q->s; p++) {
        if (q->pixels[p] < 0 || q->pixels[p] >= H0) return -1;
        for (int r = 0; r < p; r++) if (q->pixels[r] == q->pixels[p]) return -1;
    }
    uint64_t n = orc_space_size(q->s, q->k);
    if (n == 0) return -1;
    uint64_t lo = q->lo, hi = q->hi ? q->hi : n;
    if (hi > n || lo > hi) return -1;
    q->n_points = hi - lo;

    int total = orc_total_neurons(L, net->dims);
    int hmax = 0;
    for (int l = 0; l <= L; l++) if (net->dims[l] > hmax) hmax = net->dims[l];
    double *x = (double *)malloc(sizeof(double) * H0);
    double *ub = (double *)malloc(sizeof(double) * total);
    double *h0 = (double *)malloc(sizeof(double) * hmax);
    double *h1 = (double *)malloc(sizeof(double) * hmax);
    /* The unperturbed image is the point whose steps are all zero. */
    for (int j = 0; j < H0; j++) x[j] = (double)q->image[j] / 255.0;
    orc_forward(net, x, ub, h0, h1);
    q->D = orc_argmax(ub + (total - HL), HL);
    q->base_margin = q->property == 1 ? orc_threshold_margin(ub + (total - HL), HL, q->D, q->V)
                                      : orc_margin(ub + (total - HL), HL, q->D);
    free(x); free(h0); free(h1);

    if (nthreads < 1) nthreads = 1;
    size_t flip_words = ((size_t)total + 31) / 32;
    size_t ss_words = (size_t)((orc_ss_bits(L, net->dims) + 31) / 32);
    uint64_t base = lo & ~UINT64_C(31);
    uint64_t span = hi - base;
    uint64_t chunk = (span + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    chunk = (chunk + 31) & ~UINT64_C(31);
    if (chunk == 0) chunk = 32;

    orc_work *ws = (orc_work *)calloc((size_t)nthreads, sizeof(orc_work));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int i = 0; i < nthreads; i++) {
        orc_work *w = &ws[i];
        w->net = net; w->q = q; w->u_base = ub; w->D = q->D;
        uint64_t a = base + (uint64_t)i * chunk, b = a + chunk;
        if (a < lo) a = lo;
        if (a > hi) a = hi;
        if (b > hi) b = hi;
        if (b < a) b = a;
        w->a = a; w->b = b;
        if (q->flip) {
            w->flip = (uint32_t *)calloc(flip_words, 4);
            w->flip_tie = (uint32_t *)calloc(flip_words, 4);
            w->ss = (uint32_t *)calloc(ss_words ? ss_words : 1, 4);
            w->ss_tie = (uint32_t *)calloc(ss_words ? ss_words : 1, 4);
        }
        pthread_create(&th[i], NULL, orc_worker, w);
    }
    q->n_adv = 0; q->n_ties = 0; q->first_witness = UINT64_MAX;
    q->n_points = 0;
    uint64_t tl = 0;
    for (int i = 0; i < nthreads; i++) {
        pthread_join(th[i], NULL);
        orc_work *w = &ws[i];
        q->n_points += w->n_points;
        q->n_adv += w->n_adv;
        q->n_ties += w->n_ties;
        if (w->first < q->first_witness) q->first_witness = w->first;
        for (uint64_t e = 0; e < w->ties_len; e++)
            if (tl < q->ties_cap) q->ties[tl++] = w->ties[e];
        if (q->flip) {
            for (size_t e = 0; e < flip_words; e++) {
                q->flip[e] |= w->flip[e];
                q->flip_tie[e] |= w->flip_tie[e];
            }
            for (size_t e = 0; e < ss_words; e++) {
                q->ss[e] |= w->ss[e];
                q->ss_tie[e] |= w->ss_tie[e];
            }
            free(w->flip); free(w->flip_tie); free(w->ss); free(w->ss_tie);
        }
        free(w->ties);
    }
    free(ws); free(th); free(ub);
    return 0;
}

/* One point: activation potentials of every layer (u_all, length sum H_l),
 * the class D of the unperturbed image, the margin and the verdict. */
int orc_eval_point(const orc_net *net, const uint8_t *image, int s, const int *pixels, int k,
                   uint64_t t, double *u_all, int *D_out, double *margin, int *adversarial)
{
    int L = net->L, H0 = net->dims[0], HL = net->dims[L];
    int total = orc_total_neurons(L, net->dims);
    int hmax = 0;
    for (int l = 0; l <= L; l++) if (net->dims[l] > hmax) hmax = net->dims[l];
    double *x = (double *)malloc(sizeof(double) * H0);
    double *ub = (double *)malloc(sizeof(double) * total);
    double *h0 = (double *)malloc(sizeof(double) * hmax);
    double *h1 = (double *)malloc(sizeof(double) * hmax);
    for (int j = 0; j < H0; j++) x[j] = (double)image[j] / 255.0;
    orc_forward(net, x, ub, h0, h1);
    int D = orc_argmax(ub + (total - HL), HL);
    orc_point_image(net, image, s, pixels, k, t, x);
    orc_forward(net, x, u_all, h0, h1);
    const double *y = u_all + (total - HL);
    if (D_out) *D_out = D;
    if (margin) *margin = orc_margin(y, HL, D);
    if (adversarial) *adversarial = orc_argmax(y, HL) != D;
    free(x); free(ub); free(h0); free(h1);
    return 0;
}
