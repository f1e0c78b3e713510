/*
 * oracle.c - plain, slow, sequential CPU oracle for weighted random sampling
 * with alias tables ("Weighted Random Sampling on GPUs", Lehmann,
 * Huebschle-Schneider, Sanders, arXiv 2106.12270).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may use it.  It shares no code, header, table
 * or constant generator with the CUDA library; the only thing both sides see
 * is the seeded input arrays.
 *
 * Everything here is double precision (FP64) and sequential, written so that
 * each function can be checked against the paper by eye:
 *
 *   orc_exact_sum         W = sum w_i exactly, rounded once to FP64
 *                         (Sec. 1 defines W; the paper is silent on how it
 *                         is summed -- exact summation is our reading).
 *   orc_classify          light iff w_i <= W/N, heavy otherwise; the lists
 *                         l and h keep index order (Sec. 2.2, Sec. 4.2).
 *   orc_vose              Vose's sequential construction (Sec. 2.2).
 *   orc_prefix            prefix sums of light and heavy weights (Sec. 2.2).
 *   orc_split_binary      the PSA split: binary search over the prefix sums
 *                         for the Vose state after k buckets (Sec. 2.2,
 *                         Sec. 4.1 "baseline").
 *   orc_split_pary        the same splits found with partial p-ary search
 *                         (Sec. 4.1, Algorithm 1).
 *   orc_pary_search       Algorithm 1 on a plain sorted list (Sec. 4.1).
 *   orc_psa               PSA: split + sweep-pack of each section (Sec. 2.2,
 *                         Sec. 4.2).
 *   orc_psa_prec          the same PSA with its prefix arithmetic rounded to
 *                         FP64, paired FP32 or FP32 (precision study).
 *   orc_psa_plus          PSA+ (Sec. 4 "PSA+"): greedy packing per partition
 *                         tile, then PSA on the unfinished items.
 *   orc_mass              reconstructed mass of each item from a table
 *                         (Sec. 2.2: every row is one bucket of W/N).
 *   orc_philox4x32_10     Philox-4x32-10 counter-based generator (Salmon,
 *                         Moraes, Dror, Shaw, SC'11); not in the paper.
 *   orc_sample_naive      Walker's sampling (Sec. 2.2, Sec. 5 "baseline"),
 *                         integer form driven by Philox counters.
 *   orc_sample_sectioned  sampling inside equal-probability sections given
 *                         per-section counts (Sec. 5).
 *
 * Units: the oracle works in weight units (a bucket holds W/N) except where
 * a normalised value v_i = w_i / (W/N) is named (a bucket holds 1).
 *
 * All functions return 0 on success and a negative code on bad input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_EZEROSUM (-2)
#define ORC_ENONFINITE (-3)
#define ORC_ENOMEM (-4)

/* ------------------------------------------------------------------------ */
/* Exact summation of FP32 weights.                                          */
/* ------------------------------------------------------------------------ */

/* A non-negative big integer in 32-bit limbs, least significant first.  The
 * unit of the lowest bit is 2^-149, the smallest FP32 subnormal, so every
 * FP32 value is an integer in these units. */
#define BIG_LIMBS 12

static void big_add_u64_shifted(uint32_t *big, uint64_t v, unsigned shift)
{
    /* big += v << shift */
    unsigned limb = shift / 32, bit = shift % 32;
    unsigned __int128 x = (unsigned __int128)v << bit;
    uint64_t carry = 0;
    for (unsigned k = limb; k < BIG_LIMBS; ++k) {
        uint64_t part = (uint64_t)(uint32_t)(x & 0xffffffffu);
        x >>= 32;
        uint64_t s = (uint64_t)big[k] + part + carry;
        big[k] = (uint32_t)s;
        carry = s >> 32;
        if (x == 0 && carry == 0)
            break;
    }
}

static int big_bit(const uint32_t *big, int pos)
{
    if (pos < 0)
        return 0;
    return (big[pos / 32] >> (pos % 32)) & 1u;
}

static int big_top_bit(const uint32_t *big)
{
    for (int k = BIG_LIMBS - 1; k >= 0; --k)
        if (big[k])
            for (int b = 31; b >= 0; --b)
                if ((big[k] >> b) & 1u)
                    return 32 * k + b;
    return -1;
}

static int big_any_below(const uint32_t *big, int pos)
{
    /* any set bit strictly below position pos */
    for (int p = 0; p < pos; ++p)
        if (big_bit(big, p))
            return 1;
    return 0;
}

/* Round big * 2^-149 to the nearest FP64, ties to even. */
static double big_to_double(const uint32_t *big)
{
    int top = big_top_bit(big);
    if (top < 0)
        return 0.0;
    uint64_t mant = 0;
    if (top <= 52) {
        /* fewer than 54 significant bits: exact */
        for (int p = top; p >= 0; --p)
            mant = (mant << 1) | (uint64_t)big_bit(big, p);
        return ldexp((double)mant, -149);
    }
    int lsb = top - 52; /* position of the last kept bit */
    for (int p = top; p >= lsb; --p)
        mant = (mant << 1) | (uint64_t)big_bit(big, p);
    int half = big_bit(big, lsb - 1);
    int sticky = big_any_below(big, lsb - 1);
    if (half && (sticky || (mant & 1u)))
        mant += 1; /* may become 2^53: still exact in a double */
    return ldexp((double)mant, lsb - 149);
}

/* W = sum of w[0..n) computed exactly and rounded once to FP64.
 * Rejects negative, NaN and infinite weights. */
int orc_exact_sum(const float *w, uint64_t n, double *W_out)
{
    /* per biased exponent: sum of integer significands */
    uint64_t bins[256];
    memset(bins, 0, sizeof bins);
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &w[i], 4);
        uint32_t e = (u >> 23) & 0xffu, f = u & 0x7fffffu;
        if (e == 0xffu)
            return ORC_ENONFINITE;
        if ((u >> 31) && (u & 0x7fffffffu))
            return ORC_EINVAL;
        if (e == 0)
            bins[1] += f;              /* subnormal: f * 2^-149 */
        else
            bins[e] += f | 0x800000u;  /* normal: (1.f) * 2^(e-150) */
    }
    uint32_t big[BIG_LIMBS];
    memset(big, 0, sizeof big);
    for (unsigned e = 1; e < 255; ++e)
        if (bins[e])
            big_add_u64_shifted(big, bins[e], e - 1); /* 2^(e-150) = 2^(e-1) units */
    *W_out = big_to_double(big);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Classification (Sec. 2.2): light iff w_i <= W/N.  Lists keep index order  */
/* (Sec. 4.2 says l and h are sorted by item index).                         */
/* ------------------------------------------------------------------------ */

int orc_classify(const float *w, uint64_t n, double avg, uint32_t *l,
                 uint32_t *h, uint64_t *nl_out, uint64_t *nh_out)
{
    uint64_t nl = 0, nh = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if ((double)w[i] <= avg)
            l[nl++] = (uint32_t)i;
        else
            h[nh++] = (uint32_t)i;
    }
    *nl_out = nl;
    *nh_out = nh;
    return ORC_OK;
}

static int total_and_avg(const float *w, uint64_t n, double *W, double *avg)
{
    if (n == 0 || n > 0x7fffffffull)
        return ORC_EINVAL;
    int rc = orc_exact_sum(w, n, W);
    if (rc)
        return rc;
    if (*W == 0.0)
        return ORC_EZEROSUM;
    *avg = *W / (double)n;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Vose's sequential construction (Sec. 2.2), FP64, normalised units.        */
/* ------------------------------------------------------------------------ */

/* prob[i] in [0,1] is the share of row i kept by item i; alias[i] receives
 * the rest.  Work lists are first-in-first-out queues seeded in index order;
 * a heavy item whose remaining weight drops to one bucket or less moves to
 * the light queue.  Items left when one queue runs dry keep their whole
 * bucket (prob 1, alias itself), which absorbs round-off. */
int orc_vose(const float *w, uint64_t n, double *prob, uint32_t *alias,
             uint64_t *nl_out, uint64_t *nh_out, double *W_out)
{
    double W, avg;
    int rc = total_and_avg(w, n, &W, &avg);
    if (rc)
        return rc;
    double *v = malloc(n * sizeof *v);
    uint32_t *small = malloc(n * sizeof *small);
    uint32_t *large = malloc(n * sizeof *large);
    if (!v || !small || !large) {
        free(v); free(small); free(large);
        return ORC_ENOMEM;
    }
    uint64_t s_head = 0, s_tail = 0, l_head = 0, l_tail = 0;
    for (uint64_t i = 0; i < n; ++i) {
        v[i] = (double)w[i] / avg;
        if ((double)w[i] <= avg)
            small[s_tail++] = (uint32_t)i;
        else
            large[l_tail++] = (uint32_t)i;
    }
    *nl_out = s_tail;
    *nh_out = l_tail;
    while (s_head < s_tail && l_head < l_tail) {
        uint32_t lo = small[s_head++];
        uint32_t g = large[l_head];
        prob[lo] = v[lo];
        alias[lo] = g;
        v[g] = (v[g] + v[lo]) - 1.0;
        if (v[g] <= 1.0) {
            ++l_head;
            small[s_tail++] = g; /* s_tail never exceeds n: each item enters once */
        }
    }
    while (s_head < s_tail) {
        uint32_t i = small[s_head++];
        prob[i] = 1.0;
        alias[i] = i;
    }
    while (l_head < l_tail) {
        uint32_t i = large[l_head++];
        prob[i] = 1.0;
        alias[i] = i;
    }
    if (W_out)
        *W_out = W;
    free(v); free(small); free(large);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Prefix sums (Sec. 2.2): sigma_l(i) = sum_{a<i} w[l[a]],                   */
/* sigma_h(j) = sum_{b<j} w[h[b]], FP64, sequential.  Arrays have n+1 slots. */
/* ------------------------------------------------------------------------ */

int orc_prefix(const float *w, const uint32_t *list, uint64_t len,
               double *sigma)
{
    sigma[0] = 0.0;
    for (uint64_t a = 0; a < len; ++a)
        sigma[a + 1] = sigma[a] + (double)w[list[a]];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Splits (Sec. 2.2 and Sec. 4.1).                                           */
/*                                                                           */
/* A split at bucket count k is the state Vose's sweep reaches after closing */
/* k buckets: i light items and j = k - i heavy items are closed and heavy   */
/* h[j] is partly used.  Our reading of "weights balanced": with             */
/*   f(i) = sigma_l(i) + sigma_h(k - i) - k * W/N                            */
/* the split is the smallest i in [max(0, k - nh), min(k, nl)] with          */
/* f(i) <= 0, or the upper end of that range when there is none.  The spill  */
/* is what is left of h[j]: sigma_l(i) + sigma_h(j + 1) - k * W/N (0 when    */
/* j = nh).                                                                  */
/* ------------------------------------------------------------------------ */

static int split_pred(const double *sl, uint64_t nl, const double *sh,
                      uint64_t nh, double avg, uint64_t k, uint64_t i)
{
    /* monotone predicate over all i >= 0 for fixed k: false below the valid
     * range, true at and above its upper end, f(i) <= 0 inside */
    uint64_t lo = k > nh ? k - nh : 0;
    uint64_t hi = k < nl ? k : nl;
    if (i < lo)
        return 0;
    if (i >= hi)
        return 1;
    return sl[i] + sh[k - i] - (double)k * avg <= 0.0;
}

static double split_spill(const double *sl, const double *sh, uint64_t nh,
                          double avg, uint64_t k, uint64_t i)
{
    uint64_t j = k - i;
    if (j >= nh)
        return 0.0;
    return sl[i] + sh[j + 1] - (double)k * avg;
}

/* One binary search per split (the PSA baseline, Sec. 4.1). */
int orc_split_binary(const double *sl, uint64_t nl, const double *sh,
                     uint64_t nh, double avg, const uint64_t *k,
                     uint64_t nsplit, uint64_t *i_out, uint64_t *j_out,
                     double *spill_out)
{
    for (uint64_t t = 0; t < nsplit; ++t) {
        uint64_t kk = k[t];
        uint64_t a = kk > nh ? kk - nh : 0;      /* answer >= a */
        uint64_t b = kk < nl ? kk : nl;          /* answer <= b */
        while (a < b) {
            uint64_t m = a + (b - a) / 2;
            if (split_pred(sl, nl, sh, nh, avg, kk, m))
                b = m;
            else
                a = m + 1;
        }
        i_out[t] = a;
        j_out[t] = kk - a;
        spill_out[t] = split_spill(sl, sh, nh, avg, kk, a);
    }
    return ORC_OK;
}

/* Partial p-ary search (Sec. 4.1, Algorithm 1) applied to the splits: the
 * splits are handled in groups of p consecutive ones (their answers are
 * non-decreasing in k).  Phase 1 looks at p equally spaced pivots of the
 * shared range and keeps only the part between the last pivot below every
 * answer of the group (judged with the group's first split) and the first
 * pivot at or above every answer (judged with the group's last split); it
 * repeats while the range still shrinks to at most half.  Phase 2 is an
 * ordinary binary search per split inside the shared range. */
int orc_split_pary(const double *sl, uint64_t nl, const double *sh,
                   uint64_t nh, double avg, const uint64_t *k,
                   uint64_t nsplit, uint32_t p, uint64_t *i_out,
                   uint64_t *j_out, double *spill_out)
{
    if (p < 2)
        return ORC_EINVAL;
    for (uint64_t g0 = 0; g0 < nsplit; g0 += p) {
        uint64_t g1 = g0 + p < nsplit ? g0 + p : nsplit; /* [g0, g1) */
        uint64_t kf = k[g0], kl = k[g1 - 1];
        /* every answer lies in [a, b] */
        uint64_t a = kf > nh ? kf - nh : 0;
        uint64_t b = kl < nl ? kl : nl;
        if (a > b)
            a = b;
        for (;;) {
            uint64_t width = b - a;
            if (width < p)
                break;
            uint64_t na = a, nb = b;
            for (uint32_t m = 0; m < p; ++m) {
                uint64_t s = a + (width * m) / (p - 1);
                if (!split_pred(sl, nl, sh, nh, avg, kf, s)) {
                    /* "smaller": even the first split's answer is > s */
                    if (s + 1 > na)
                        na = s + 1;
                } else if (split_pred(sl, nl, sh, nh, avg, kl, s)) {
                    /* "larger": even the last split's answer is <= s */
                    if (s < nb)
                        nb = s;
                }
            }
            if (nb < na)
                nb = na;
            uint64_t nwidth = nb - na;
            a = na;
            b = nb;
            if (2 * nwidth > width)
                break; /* the range no longer shrinks enough */
        }
        for (uint64_t t = g0; t < g1; ++t) {
            uint64_t kk = k[t];
            uint64_t lo = kk > nh ? kk - nh : 0;
            uint64_t hi = kk < nl ? kk : nl;
            uint64_t x = a > lo ? a : lo;
            uint64_t y = b < hi ? b : hi;
            if (x > y)
                x = y;
            while (x < y) {
                uint64_t m = x + (y - x) / 2;
                if (split_pred(sl, nl, sh, nh, avg, kk, m))
                    y = m;
                else
                    x = m + 1;
            }
            i_out[t] = x;
            j_out[t] = kk - x;
            spill_out[t] = split_spill(sl, sh, nh, avg, kk, x);
        }
    }
    return ORC_OK;
}

/* Algorithm 1 on a sorted list: for each key x_t (keys sorted ascending),
 * return the number of list entries <= x_t (the upper-bound position).
 * Phase 1 narrows a shared range with p pivots using only the smallest and
 * the largest key of the group; phase 2 is a binary search per key. */
int orc_pary_search(const double *list, uint64_t n, const double *keys,
                    uint64_t nkeys, uint32_t p, uint64_t *out)
{
    if (p < 2)
        return ORC_EINVAL;
    for (uint64_t g0 = 0; g0 < nkeys; g0 += p) {
        uint64_t g1 = g0 + p < nkeys ? g0 + p : nkeys;
        double xmin = keys[g0], xmax = keys[g1 - 1];
        uint64_t a = 0, b = n; /* every answer lies in [a, b] */
        for (;;) {
            uint64_t width = b - a;
            if (width < p)
                break;
            uint64_t na = a, nb = b;
            for (uint32_t m = 0; m < p; ++m) {
                uint64_t s = a + (width * m) / (p - 1);
                if (s >= n)
                    continue;
                if (list[s] <= xmin) {          /* "smaller": every answer > s */
                    if (s + 1 > na)
                        na = s + 1;
                } else if (list[s] > xmax) {    /* "larger": every answer <= s */
                    if (s < nb)
                        nb = s;
                }
            }
            if (nb < na)
                nb = na;
            uint64_t nwidth = nb - na;
            a = na;
            b = nb;
            if (2 * nwidth > width)
                break;
        }
        for (uint64_t t = g0; t < g1; ++t) {
            uint64_t x = a, y = b;
            while (x < y) {
                uint64_t m = x + (y - x) / 2;
                if (list[m] > keys[t])
                    y = m;
                else
                    x = m + 1;
            }
            out[t] = x;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* PSA (Sec. 2.2, Sec. 4.2): split into sections of S buckets, then sweep     */
/* each section from its split state.                                         */
/* ------------------------------------------------------------------------ */

/* Section t covers buckets [k_t, k_{t+1}) with k_t = min(t*S, n).  The sweep
 * keeps r, the weight left in the current heavy item h[j].  While the section
 * still has buckets to close:
 *   - if r <= W/N and the section still owns heavy items (or it has no light
 *     items left), heavy h[j] closes its own bucket: it keeps r and takes the
 *     rest from h[j+1]; then h[j+1] becomes current with its weight reduced
 *     by what it gave;
 *   - otherwise light l[i] closes its bucket with its own weight and takes
 *     the rest from h[j].
 * A bucket whose donor does not exist (no heavy item left) keeps its whole
 * bucket (prob 1, alias itself), as Vose's clean-up does.  prob is the kept
 * share of the bucket, clamped to [0,1]. */
int orc_psa(const float *w, uint64_t n, uint64_t S, double *prob,
            uint32_t *alias, uint64_t *nl_out, uint64_t *nh_out,
            uint64_t *split_i, uint64_t *split_j, double *split_spill_out,
            uint32_t pary_p)
{
    double W, avg;
    int rc = total_and_avg(w, n, &W, &avg);
    if (rc)
        return rc;
    if (S == 0)
        return ORC_EINVAL;
    uint32_t *l = malloc(n * sizeof *l), *h = malloc(n * sizeof *h);
    double *sl = malloc((n + 1) * sizeof *sl), *sh = malloc((n + 1) * sizeof *sh);
    uint64_t nsec = (n + S - 1) / S;
    uint64_t *k = malloc((nsec + 1) * sizeof *k);
    uint64_t *si = malloc((nsec + 1) * sizeof *si), *sj = malloc((nsec + 1) * sizeof *sj);
    double *sp = malloc((nsec + 1) * sizeof *sp);
    if (!l || !h || !sl || !sh || !k || !si || !sj || !sp) {
        rc = ORC_ENOMEM;
        goto out;
    }
    uint64_t nl, nh;
    orc_classify(w, n, avg, l, h, &nl, &nh);
    orc_prefix(w, l, nl, sl);
    orc_prefix(w, h, nh, sh);
    for (uint64_t t = 0; t <= nsec; ++t)
        k[t] = t * S < n ? t * S : n;
    if (pary_p >= 2)
        orc_split_pary(sl, nl, sh, nh, avg, k, nsec + 1, pary_p, si, sj, sp);
    else
        orc_split_binary(sl, nl, sh, nh, avg, k, nsec + 1, si, sj, sp);
    for (uint64_t t = 0; t < nsec; ++t) {
        uint64_t i = si[t], j = sj[t];
        uint64_t i_end = si[t + 1], j_end = sj[t + 1];
        double r = sp[t]; /* weight left in h[j] */
        while (i < i_end || j < j_end) {
            int light_left = i < i_end;
            int heavy_left = j < j_end;
            if (heavy_left && (r <= avg || !light_left)) {
                uint32_t g = h[j];
                double keep = r / avg;
                prob[g] = keep < 0.0 ? 0.0 : (keep > 1.0 ? 1.0 : keep);
                if (j + 1 < nh) {
                    alias[g] = h[j + 1];
                    r = r + (double)w[h[j + 1]] - avg;
                } else {
                    prob[g] = 1.0;
                    alias[g] = g;
                    r = 0.0;
                }
                ++j;
            } else {
                uint32_t lo = l[i];
                if (j < nh) {
                    prob[lo] = (double)w[lo] / avg;
                    alias[lo] = h[j];
                    r = r - (avg - (double)w[lo]);
                } else {
                    prob[lo] = 1.0;
                    alias[lo] = lo;
                }
                ++i;
            }
        }
    }
    *nl_out = nl;
    *nh_out = nh;
    if (split_i)
        for (uint64_t t = 0; t <= nsec; ++t) {
            split_i[t] = si[t];
            split_j[t] = sj[t];
            split_spill_out[t] = sp[t];
        }
    rc = ORC_OK;
out:
    free(l); free(h); free(sl); free(sh); free(k); free(si); free(sj); free(sp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* PSA+ (Sec. 4 "PSA+"): greedy packing inside each partition tile, then PSA  */
/* on the items the greedy step did not finish.                              */
/*                                                                           */
/* Tile t holds items [tT, min((t+1)T, n)).  If it has at least m light and  */
/* m heavy items, its lights and heavies (index order) are swept as in PSA:   */
/* the current heavy with r left closes its own bucket when r <= W/N and the  */
/* tile has a next heavy; otherwise it fills the next light bucket.  The     */
/* sweep stops when the tile has no light left to fill or no next heavy.     */
/* The heavy current at that point keeps its remaining weight r and, like   */
/* every other item not yet closed, goes to the rest of the build: light iff */
/* its current weight is <= W/N.  That rest is built by the PSA above (binary */
/* split search, sections of S buckets) on the current weights, in index    */
/* order.  Reading of the paper: the leftover heavy's weight and its class  */
/* are not stated; carrying r is what keeps every bucket at W/N.            */
/* ------------------------------------------------------------------------ */

/* PSA over a list of items (ids, current weights), lights and heavies given
 * in index order; the arithmetic of orc_psa with the binary split. */
static int psa_rest(const uint32_t *lid, const double *lw, uint64_t nl,
                    const uint32_t *hid, const double *hw, uint64_t nh,
                    double avg, uint64_t S, double *prob, uint32_t *alias)
{
    const uint64_t n = nl + nh;
    if (n == 0)
        return ORC_OK;
    double *sl = malloc((nl + 1) * sizeof *sl), *sh = malloc((nh + 1) * sizeof *sh);
    if (!sl || !sh) {
        free(sl); free(sh);
        return ORC_ENOMEM;
    }
    sl[0] = sh[0] = 0.0;
    for (uint64_t a = 0; a < nl; ++a)
        sl[a + 1] = sl[a] + lw[a];
    for (uint64_t b = 0; b < nh; ++b)
        sh[b + 1] = sh[b] + hw[b];
    const uint64_t nsec = (n + S - 1) / S;
    uint64_t i_prev = 0, j_prev = 0;
    double sp_prev = nh ? sl[0] + sh[1] - 0.0 : 0.0;
    for (uint64_t t = 1; t <= nsec; ++t) {
        /* the split at k = min(tS, n) */
        uint64_t kk = t * S < n ? t * S : n;
        uint64_t a = kk > nh ? kk - nh : 0, b = kk < nl ? kk : nl;
        while (a < b) {
            uint64_t m = a + (b - a) / 2;
            if (sl[m] + sh[kk - m] - (double)kk * avg <= 0.0)
                b = m;
            else
                a = m + 1;
        }
        const uint64_t i_end = a, j_end = kk - a;
        const double sp = j_end < nh ? sl[a] + sh[j_end + 1] - (double)kk * avg : 0.0;
        /* sweep section t-1 from the previous split */
        uint64_t i = i_prev, j = j_prev;
        double r = sp_prev;
        while (i < i_end || j < j_end) {
            int light_left = i < i_end;
            int heavy_left = j < j_end;
            if (heavy_left && (r <= avg || !light_left)) {
                uint32_t g = hid[j];
                double keep = r / avg;
                prob[g] = keep < 0.0 ? 0.0 : (keep > 1.0 ? 1.0 : keep);
                if (j + 1 < nh) {
                    alias[g] = hid[j + 1];
                    r = r + hw[j + 1] - avg;
                } else {
                    prob[g] = 1.0;
                    alias[g] = g;
                    r = 0.0;
                }
                ++j;
            } else {
                uint32_t lo = lid[i];
                if (j < nh) {
                    prob[lo] = lw[i] / avg;
                    alias[lo] = hid[j];
                    r = r - (avg - lw[i]);
                } else {
                    prob[lo] = 1.0;
                    alias[lo] = lo;
                }
                ++i;
            }
        }
        i_prev = i_end;
        j_prev = j_end;
        sp_prev = sp;
    }
    free(sl); free(sh);
    return ORC_OK;
}

int orc_psa_plus(const float *w, uint64_t n, uint64_t S, uint64_t T,
                 uint64_t m, double *prob, uint32_t *alias, uint64_t *greedy)
{
    double W, avg;
    int rc = total_and_avg(w, n, &W, &avg);
    if (rc)
        return rc;
    if (S == 0 || T == 0)
        return ORC_EINVAL;
    /* the rest: ids and current weights, lights and heavies in index order */
    uint32_t *lid = malloc(n * sizeof *lid), *hid = malloc(n * sizeof *hid);
    double *lw = malloc(n * sizeof *lw), *hw = malloc(n * sizeof *hw);
    uint32_t *tl = malloc(T * sizeof *tl), *th = malloc(T * sizeof *th);
    double *cur = malloc(n * sizeof *cur);
    unsigned char *done = calloc(n, 1);
    if (!lid || !hid || !lw || !hw || !tl || !th || !cur || !done) {
        rc = ORC_ENOMEM;
        goto out;
    }
    uint64_t closed = 0;
    for (uint64_t i = 0; i < n; ++i)
        cur[i] = (double)w[i];
    for (uint64_t t0 = 0; t0 < n; t0 += T) {
        const uint64_t t1 = t0 + T < n ? t0 + T : n;
        uint64_t ntl = 0, nth = 0;
        for (uint64_t i = t0; i < t1; ++i) {
            if ((double)w[i] <= avg)
                tl[ntl++] = (uint32_t)i;
            else
                th[nth++] = (uint32_t)i;
        }
        if (ntl < m || nth < m || ntl == 0 || nth == 0)
            continue;
        uint64_t i = 0, j = 0;
        double r = (double)w[th[0]];
        for (;;) {
            if (r <= avg) {
                if (j + 1 >= nth)
                    break;               /* no next heavy in the tile */
                uint32_t g = th[j];
                double keep = r / avg;
                prob[g] = keep < 0.0 ? 0.0 : (keep > 1.0 ? 1.0 : keep);
                alias[g] = th[j + 1];
                done[g] = 1;
                ++closed;
                r = r + (double)w[th[j + 1]] - avg;
                ++j;
            } else {
                if (i >= ntl)
                    break;               /* no light left to fill */
                uint32_t lo = tl[i];
                prob[lo] = (double)w[lo] / avg;
                alias[lo] = th[j];
                done[lo] = 1;
                ++closed;
                r = r - (avg - (double)w[lo]);
                ++i;
            }
        }
        cur[th[j]] = r;                  /* the heavy left current */
    }
    uint64_t nl = 0, nh = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (done[i])
            continue;
        if (cur[i] <= avg) {
            lid[nl] = (uint32_t)i;
            lw[nl++] = cur[i];
        } else {
            hid[nh] = (uint32_t)i;
            hw[nh++] = cur[i];
        }
    }
    rc = psa_rest(lid, lw, nl, hid, hw, nh, avg, S, prob, alias);
    if (greedy)
        *greedy = closed;
out:
    free(lid); free(hid); free(lw); free(hw); free(tl); free(th); free(cur); free(done);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* PSA in a chosen working precision (precision study).                      */
/*                                                                           */
/* The paper keeps the prefix sums, the split comparisons and the sweep's     */
/* residual in FP64 (Sec. 2.2, Sec. 6).  This copy of the PSA above (binary   */
/* split search) rounds every one of those quantities to a working precision */
/* after each operation:                                                      */
/*   prec 0: FP64 (no extra rounding; equal to orc_psa bit for bit),          */
/*   prec 1: a pair of FP32 values hi + lo (about 48 significant bits: what  */
/*           compensated FP32 summation keeps),                               */
/*   prec 2: plain FP32.                                                      */
/* The total W, the average and the light/heavy classification are exact as  */
/* in orc_psa, so only the prefix arithmetic differs.                         */
/* ------------------------------------------------------------------------ */

static double wp(int prec, double x)
{
    if (prec == 1) {
        float hi = (float)x;
        float lo = (float)(x - (double)hi);
        return (double)hi + (double)lo;
    }
    if (prec == 2)
        return (double)(float)x;
    return x;
}

int orc_psa_prec(const float *w, uint64_t n, uint64_t S, int prec,
                 double *prob, uint32_t *alias)
{
    double W, avg0;
    int rc = total_and_avg(w, n, &W, &avg0);
    if (rc)
        return rc;
    if (S == 0 || prec < 0 || prec > 2)
        return ORC_EINVAL;
    const double avg = wp(prec, avg0);
    uint32_t *l = malloc(n * sizeof *l), *h = malloc(n * sizeof *h);
    double *sl = malloc((n + 1) * sizeof *sl), *sh = malloc((n + 1) * sizeof *sh);
    uint64_t nsec = (n + S - 1) / S;
    uint64_t *si = malloc((nsec + 1) * sizeof *si), *sj = malloc((nsec + 1) * sizeof *sj);
    double *sp = malloc((nsec + 1) * sizeof *sp);
    if (!l || !h || !sl || !sh || !si || !sj || !sp) {
        rc = ORC_ENOMEM;
        goto out;
    }
    uint64_t nl, nh;
    orc_classify(w, n, avg0, l, h, &nl, &nh);
    sl[0] = sh[0] = 0.0;
    for (uint64_t a = 0; a < nl; ++a)
        sl[a + 1] = wp(prec, sl[a] + (double)w[l[a]]);
    for (uint64_t b = 0; b < nh; ++b)
        sh[b + 1] = wp(prec, sh[b] + (double)w[h[b]]);
    /* splits: the smallest i with f(i) = sl(i) + sh(k-i) - k avg <= 0 in the
     * valid range, each term rounded to the working precision */
    for (uint64_t t = 0; t <= nsec; ++t) {
        uint64_t kk = t * S < n ? t * S : n;
        uint64_t a = kk > nh ? kk - nh : 0, b = kk < nl ? kk : nl;
        double kavg = wp(prec, (double)kk * avg);
        while (a < b) {
            uint64_t m = a + (b - a) / 2;
            if (wp(prec, wp(prec, sl[m] + sh[kk - m]) - kavg) <= 0.0)
                b = m;
            else
                a = m + 1;
        }
        si[t] = a;
        sj[t] = kk - a;
        sp[t] = kk - a < nh ? wp(prec, wp(prec, sl[a] + sh[kk - a + 1]) - kavg) : 0.0;
    }
    for (uint64_t t = 0; t < nsec; ++t) {
        uint64_t i = si[t], j = sj[t];
        uint64_t i_end = si[t + 1], j_end = sj[t + 1];
        double r = sp[t];
        while (i < i_end || j < j_end) {
            int light_left = i < i_end;
            int heavy_left = j < j_end;
            if (heavy_left && (r <= avg || !light_left)) {
                uint32_t g = h[j];
                double keep = wp(prec, r / avg);
                prob[g] = keep < 0.0 ? 0.0 : (keep > 1.0 ? 1.0 : keep);
                if (j + 1 < nh) {
                    alias[g] = h[j + 1];
                    r = wp(prec, wp(prec, r + (double)w[h[j + 1]]) - avg);
                } else {
                    prob[g] = 1.0;
                    alias[g] = g;
                    r = 0.0;
                }
                ++j;
            } else {
                uint32_t lo = l[i];
                if (j < nh) {
                    prob[lo] = wp(prec, (double)w[lo] / avg);
                    alias[lo] = h[j];
                    r = wp(prec, r - wp(prec, avg - (double)w[lo]));
                } else {
                    prob[lo] = 1.0;
                    alias[lo] = lo;
                }
                ++i;
            }
        }
    }
    rc = ORC_OK;
out:
    free(l); free(h); free(sl); free(sh); free(si); free(sj); free(sp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Reconstructed mass (Sec. 2.2): row b keeps prob[b] of its bucket for item  */
/* b and gives 1 - prob[b] to alias[b]; an exact table gives item i the mass */
/* N * w_i / W buckets.                                                       */
/* ------------------------------------------------------------------------ */

int orc_mass(const double *prob, const uint32_t *alias, uint64_t n,
             double *mass)
{
    for (uint64_t i = 0; i < n; ++i)
        mass[i] = 0.0;
    for (uint64_t b = 0; b < n; ++b) {
        if (alias[b] >= n)
            return ORC_EINVAL;
        mass[b] += prob[b];
        mass[alias[b]] += 1.0 - prob[b];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al., SC'11): a 4x32-bit counter and a 2x32-bit   */
/* key; ten rounds, each multiplying words 0 and 2 by fixed odd constants,    */
/* mixing the high halves with words 1, 3 and the round key, and advancing    */
/* the key by fixed Weyl increments.                                          */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * x0;
        uint64_t p1 = (uint64_t)mul1 * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Sampling (Sec. 2.2, Sec. 5).                                               */
/*                                                                            */
/* Walker's rule draws U, takes the integer part of U*N as the row and       */
/* compares the fractional part with the row's kept share.  Integer form     */
/* used here: one Philox call gives two 64-bit values u; for each,           */
/*   P = u * N (a 128-bit product), row = P >> 64 (integer part of U*N),     */
/*   coin = bits 32..63 of P (top 32 bits of the fractional part),           */
/*   output row if coin < ceil(prob[row] * 2^32), else alias[row].           */
/* Sample q of a request uses call c = q / 2 (first or second half by q % 2) */
/* with counter (c_lo, c_hi, stream_lo, stream_hi) and key (seed_lo,         */
/* seed_hi).                                                                  */
/* ------------------------------------------------------------------------ */

static uint64_t coin_threshold(float p)
{
    /* ceil(p * 2^32) for p in [0,1]; exact: the product is exact in FP64 */
    double t = ceil((double)p * 4294967296.0);
    if (t < 0.0)
        t = 0.0;
    if (t > 4294967296.0)
        t = 4294967296.0;
    return (uint64_t)t;
}

static uint32_t walker_pick(uint64_t u, uint64_t rows, uint64_t base,
                            const float *prob, const uint32_t *alias)
{
    unsigned __int128 P = (unsigned __int128)u * rows;
    uint64_t row = base + (uint64_t)(P >> 64);
    uint32_t coin = (uint32_t)(P >> 32);
    return (uint64_t)coin < coin_threshold(prob[row]) ? (uint32_t)row
                                                      : alias[row];
}

static uint64_t half_of(const uint32_t x[4], uint64_t q)
{
    return (q & 1u) ? ((uint64_t)x[2] << 32 | x[3]) : ((uint64_t)x[0] << 32 | x[1]);
}

int orc_sample_naive(const float *prob, const uint32_t *alias, uint64_t n,
                     uint64_t first, uint64_t count, uint64_t seed,
                     uint32_t stream_lo, uint32_t stream_hi, uint32_t *out)
{
    if (n == 0)
        return ORC_EINVAL;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint64_t t = 0; t < count; ++t) {
        uint64_t q = first + t, c = q >> 1;
        uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), stream_lo, stream_hi};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        out[t] = walker_pick(half_of(x, q), n, 0, prob, alias);
    }
    return ORC_OK;
}

/* Sectioned sampling (Sec. 5): the rows are cut into nsec contiguous sections
 * of near-equal size, section s covering rows [floor(s*n/nsec),
 * floor((s+1)*n/nsec)).  Given how many samples each section draws (counts,
 * in section order), sample q of section s uses the counter (c_lo, c_hi, s,
 * tag) with c = q / 2 and picks a row inside the section by Walker's rule.
 * Samples are written section by section, in order. */
int orc_sample_sectioned(const float *prob, const uint32_t *alias, uint64_t n,
                         uint64_t nsec, const uint64_t *counts, uint64_t seed,
                         uint32_t tag, uint32_t *out)
{
    if (n == 0 || nsec == 0 || nsec > n)
        return ORC_EINVAL;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t pos = 0;
    for (uint64_t s = 0; s < nsec; ++s) {
        uint64_t r0 = (uint64_t)(((unsigned __int128)s * n) / nsec);
        uint64_t r1 = (uint64_t)(((unsigned __int128)(s + 1) * n) / nsec);
        for (uint64_t q = 0; q < counts[s]; ++q) {
            uint64_t c = q >> 1;
            uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), (uint32_t)s, tag};
            uint32_t x[4];
            orc_philox4x32_10(ctr, key, x);
            out[pos++] = walker_pick(half_of(x, q), r1 - r0, r0, prob, alias);
        }
    }
    return ORC_OK;
}
