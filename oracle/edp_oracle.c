/*
 * edp_oracle.c -- plain CPU oracle for the EDP / RMS method of
 * M. G. Mozerov, "Extended Dynamic Programming and Fast Multidimensional
 * Search Algorithm for Energy Minimization in Stereo and Motion"
 * (arXiv 1410.7922).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Everything is exact integer arithmetic held in int64.  Every value that
 * the GPU path keeps in int32 (costs, sums, messages, partial sums) is
 * checked to fit in int32 and ORACLE_ERR_RANGE is returned otherwise.
 *
 * Two tiers compute the min-search operator M (Eq. M_strf):
 *   tier 0  "brute"  the definition, M(S)(q) = min_q' S(q') + V(q',q),
 *                    O(Q^2) per message (the paper's SFMS, Sec. 3 / Table 1);
 *   tier 1  "rms"    the paper's recursive minimum search: per label axis the
 *                    two-sweep operator L_r of Eq. L_dec3 / L_dec5 / L_dec6 for
 *                    the truncated linear prior (LRMS), or the per-axis
 *                    windowed operator of Eq. M_decmp (GRMS) for l1 = 2,
 *                    followed by the clip of Eq. derivation1.
 * Tier 1 is only trusted because the tests check it against tier 0.
 *
 * Label space: R axes (1..3) with Q[r] labels each, axis 0 fastest;
 * linear label q = q0 + Q0*(q1 + Q1*q2).  Label coordinate q_r maps to the
 * displacement vmin[r] + step[r]*q_r (step = +1 or -1), the affine rescale
 * the paper allows below Eq. v_r_x_d.  Axis 0 displaces x into I1, axis 1
 * displaces y into I1, axis 2 (R = 3 only) displaces x into a third image I2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_RANGE 2
#define ORACLE_ERR_NOMEM 3

#define PRIOR_JOINT 0    /* lambda * min(sum_r |d_r|^l1, g^l1)   Eq. Smooth_value_t */
#define PRIOR_PER_AXIS 1 /* sum_r lambda * min(|d_r|^l1, g^l1)  separable variant  */

#define COST_PAIR 0      /* Eq. Cost_value with I1                                   */
#define COST_PAIR_STEREO3 1 /* R = 3: |I1(x+o0,y+o1)-I0|^l2 + |I2(x+o2,y)-I0|^l2, cut */
#define COST_COMPOSITE 2 /* Eq. Cost_cmp: C_{I0->I1}(x, v) ^ C_{I0->I2}(x, -v)       */

#define INF64 ((int64_t)1 << 60)

typedef struct {
    int32_t R;
    int32_t Q[3];
    int32_t lambda;
    int32_t g;
    int32_t l1;
    int32_t mode;
} oracle_prior_t;

static int fits32(int64_t v) { return v >= INT32_MIN && v <= INT32_MAX; }

static int64_t ipow(int64_t a, int e) { return e == 1 ? a : a * a; }

static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

/* floor(s / 2) for any sign: the 1/D factor of Eq. DP_2D_1 with D = 2 on
 * integers (C division truncates toward zero, so negative odd values need
 * one more step down). */
static int64_t floor_half(int64_t s) { return s >= 0 ? s / 2 : (s - 1) / 2; }

static int64_t total_labels(const oracle_prior_t *p) {
    int64_t Q = 1;
    for (int r = 0; r < p->R; ++r) Q *= p->Q[r];
    return Q;
}

static void decode(const oracle_prior_t *p, int64_t q, int64_t c[3]) {
    c[0] = c[1] = c[2] = 0;
    for (int r = 0; r < p->R; ++r) {
        c[r] = q % p->Q[r];
        q /= p->Q[r];
    }
}

static int check_prior(const oracle_prior_t *p) {
    if (p->R < 1 || p->R > 3) return ORACLE_ERR_ARG;
    for (int r = 0; r < p->R; ++r)
        if (p->Q[r] < 1) return ORACLE_ERR_ARG;
    if (p->lambda < 0 || p->g < 1 || (p->l1 != 1 && p->l1 != 2)) return ORACLE_ERR_ARG;
    if (p->mode != PRIOR_JOINT && p->mode != PRIOR_PER_AXIS) return ORACLE_ERR_ARG;
    return ORACLE_OK;
}

/* V(q, q'): the truncated smoothness term of Eq. Smooth_value_t for one edge.
 * JOINT truncates the sum over the R label axes (the paper's form); PER_AXIS
 * truncates each axis separately. */
int64_t oracle_prior(const oracle_prior_t *p, int64_t q, int64_t qp) {
    int64_t a[3], b[3];
    decode(p, q, a);
    decode(p, qp, b);
    int64_t cap = ipow(p->g, p->l1);
    if (p->mode == PRIOR_JOINT) {
        int64_t f = 0;
        for (int r = 0; r < p->R; ++r) f += ipow(iabs64(a[r] - b[r]), p->l1);
        return (int64_t)p->lambda * (f < cap ? f : cap);
    }
    int64_t v = 0;
    for (int r = 0; r < p->R; ++r) {
        int64_t f = ipow(iabs64(a[r] - b[r]), p->l1);
        v += (int64_t)p->lambda * (f < cap ? f : cap);
    }
    return v;
}

/* ------------------------------------------------------------------------ */
/* Cost volume, Eq. Cost_value: C(x, v) = |I1(x + v) - I0(x)|^l2 ^ Cmax.      */
/* A displaced pixel outside the image costs Cmax.                            */
/* ------------------------------------------------------------------------ */

static int64_t pixel_cost(const uint8_t *I0, const uint8_t *I1, int W, int H, int x, int y,
                          int64_t dx, int64_t dy, int l2, int64_t cmax, int *oob) {
    int64_t xs = x + dx, ys = y + dy;
    if (xs < 0 || xs >= W || ys < 0 || ys >= H) {
        *oob = 1;
        return cmax;
    }
    *oob = 0;
    int64_t d = (int64_t)I1[ys * W + xs] - (int64_t)I0[(int64_t)y * W + x];
    return ipow(iabs64(d), l2);
}

static int64_t cost_at(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H,
                       int x, int y, const int64_t o[3], int R, int l2, int64_t cmax,
                       int cost_mode) {
    int oob;
    if (cost_mode == COST_PAIR) {
        int64_t c = pixel_cost(I0, I1, W, H, x, y, o[0], R >= 2 ? o[1] : 0, l2, cmax, &oob);
        return c < cmax ? c : cmax;
    }
    if (cost_mode == COST_PAIR_STEREO3) {
        int oob2;
        int64_t c1 = pixel_cost(I0, I1, W, H, x, y, o[0], o[1], l2, cmax, &oob);
        int64_t c2 = pixel_cost(I0, I2, W, H, x, y, o[2], 0, l2, cmax, &oob2);
        if (oob || oob2) return cmax;
        int64_t c = c1 + c2;
        return c < cmax ? c : cmax;
    }
    /* COST_COMPOSITE: each term truncated by Eq. Cost_value, then the min. */
    int oob2;
    int64_t c1 = pixel_cost(I0, I1, W, H, x, y, o[0], R >= 2 ? o[1] : 0, l2, cmax, &oob);
    int64_t c2 = pixel_cost(I0, I2, W, H, x, y, -o[0], R >= 2 ? -o[1] : 0, l2, cmax, &oob2);
    if (c1 > cmax) c1 = cmax;
    if (c2 > cmax) c2 = cmax;
    return c1 < c2 ? c1 : c2;
}

static int check_cost_args(int W, int H, int R, const int32_t *Q, const int32_t *step, int l2,
                           int cmax, int cost_mode, const uint8_t *I2) {
    if (W < 1 || H < 1 || R < 1 || R > 3 || (l2 != 1 && l2 != 2) || cmax < 0) return ORACLE_ERR_ARG;
    for (int r = 0; r < R; ++r)
        if (Q[r] < 1 || (step[r] != 1 && step[r] != -1)) return ORACLE_ERR_ARG;
    if (cost_mode == COST_PAIR && R > 2) return ORACLE_ERR_ARG;
    if (cost_mode == COST_PAIR_STEREO3 && (R != 3 || !I2)) return ORACLE_ERR_ARG;
    if (cost_mode == COST_COMPOSITE && (R > 2 || !I2)) return ORACLE_ERR_ARG;
    if (cost_mode < 0 || cost_mode > 2) return ORACLE_ERR_ARG;
    return ORACLE_OK;
}

int oracle_cost_volume(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H,
                       int R, const int32_t *Q, const int32_t *vmin, const int32_t *step, int l2,
                       int cmax, int cost_mode, int32_t *C) {
    int rc = check_cost_args(W, H, R, Q, step, l2, cmax, cost_mode, I2);
    if (rc) return rc;
    int64_t QQ = 1;
    for (int r = 0; r < R; ++r) QQ *= Q[r];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int64_t q = 0; q < QQ; ++q) {
                int64_t rest = q, o[3] = {0, 0, 0};
                for (int r = 0; r < R; ++r) {
                    o[r] = vmin[r] + (int64_t)step[r] * (rest % Q[r]);
                    rest /= Q[r];
                }
                int64_t c = cost_at(I0, I1, I2, W, H, x, y, o, R, l2, cmax, cost_mode);
                if (!fits32(c)) return ORACLE_ERR_RANGE;
                C[((int64_t)y * W + x) * QQ + q] = (int32_t)c;
            }
    return ORACLE_OK;
}

/* Cost restricted to a per-pixel box of labels (the windowed form): the box
 * of pixel x has side `win` on every axis and starts at centre - (win-1)/2,
 * where the centre (label coordinates) is clamped so the box fits. */
static void clamp_centre(const oracle_prior_t *p, int win, const int32_t *c_in, int64_t lo[3]) {
    int h = (win - 1) / 2;
    for (int r = 0; r < 3; ++r) lo[r] = 0;
    for (int r = 0; r < p->R; ++r) {
        int64_t c = c_in[r];
        if (c < h) c = h;
        if (c > p->Q[r] - 1 - h) c = p->Q[r] - 1 - h;
        lo[r] = c - h;
    }
}

int oracle_cost_window(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H,
                       int R, const int32_t *Q, const int32_t *vmin, const int32_t *step, int l2,
                       int cmax, int cost_mode, const int32_t *centre, int win, int32_t *Cw) {
    int rc = check_cost_args(W, H, R, Q, step, l2, cmax, cost_mode, I2);
    if (rc) return rc;
    if (R > 2 || win < 1 || (win & 1) == 0) return ORACLE_ERR_ARG;
    oracle_prior_t p;
    memset(&p, 0, sizeof p);
    p.R = R;
    for (int r = 0; r < R; ++r) {
        p.Q[r] = Q[r];
        if (Q[r] < win) return ORACLE_ERR_ARG;
    }
    int64_t QW = R == 1 ? win : (int64_t)win * win;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t lo[3];
            clamp_centre(&p, win, centre + ((int64_t)y * W + x) * R, lo);
            for (int64_t w = 0; w < QW; ++w) {
                int64_t o[3] = {0, 0, 0};
                int64_t wc[2] = {w % win, w / win};
                for (int r = 0; r < R; ++r) o[r] = vmin[r] + (int64_t)step[r] * (lo[r] + wc[r]);
                int64_t c = cost_at(I0, I1, I2, W, H, x, y, o, R, l2, cmax, cost_mode);
                Cw[((int64_t)y * W + x) * QW + w] = (int32_t)c;
            }
        }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Min-search operator M (Eq. M_strf):  out(q) = min_q' h(q') + V(q', q).   */
/* ------------------------------------------------------------------------ */

static void message_brute(const oracle_prior_t *p, const int64_t *h, int64_t *out) {
    int64_t Q = total_labels(p);
    for (int64_t q = 0; q < Q; ++q) {
        int64_t best = INF64;
        for (int64_t qp = 0; qp < Q; ++qp) {
            int64_t v = h[qp] + oracle_prior(p, qp, q);
            if (v < best) best = v;
        }
        out[q] = best;
    }
}

/* One label axis of the RMS: lines along axis r of the buffer `t`. */
static void axis_lines(const oracle_prior_t *p, int r, int64_t *stride, int64_t *nlines,
                       int64_t *len) {
    int64_t Q = total_labels(p);
    int64_t s = 1;
    for (int i = 0; i < r; ++i) s *= p->Q[i];
    *stride = s;
    *len = p->Q[r];
    *nlines = Q / p->Q[r];
}

static int64_t line_base(const oracle_prior_t *p, int r, int64_t line) {
    /* line enumerates all coordinates except axis r */
    int64_t s = 1;
    for (int i = 0; i < r; ++i) s *= p->Q[i];
    int64_t inner = line % s, outer = line / s;
    return inner + outer * s * p->Q[r];
}

/* L_r of Eq. L_dec6 on one line: forward sweep (Eq. L_dec3), backward sweep
 * (Eq. L_dec5), then the element-wise min of the two.  Weight lambda per
 * label step, no truncation (the clip comes afterwards). */
static void lrms_line(int64_t *v, int64_t n, int64_t stride, int64_t lambda, int64_t *fw,
                      int64_t *bw) {
    fw[0] = v[0];
    for (int64_t i = 1; i < n; ++i) {
        int64_t a = fw[i - 1] + lambda, b = v[i * stride];
        fw[i] = a < b ? a : b;
    }
    bw[n - 1] = v[(n - 1) * stride];
    for (int64_t i = n - 2; i >= 0; --i) {
        int64_t a = bw[i + 1] + lambda, b = v[i * stride];
        bw[i] = a < b ? a : b;
    }
    for (int64_t i = 0; i < n; ++i) v[i * stride] = fw[i] < bw[i] ? fw[i] : bw[i];
}

/* GRMS operator of Eq. M_decmp on one line: min over |u| < g of
 * h(v + u) + lambda * f(|u|), f(u) = u^l1. */
static void grms_line(int64_t *v, int64_t n, int64_t stride, int64_t lambda, int64_t g, int l1,
                      int64_t *tmp) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t best = INF64;
        for (int64_t u = -(g - 1); u <= g - 1; ++u) {
            int64_t j = i + u;
            if (j < 0 || j >= n) continue;
            int64_t c = v[j * stride] + lambda * ipow(iabs64(u), l1);
            if (c < best) best = c;
        }
        tmp[i] = best;
    }
    for (int64_t i = 0; i < n; ++i) v[i * stride] = tmp[i];
}

static int message_rms(const oracle_prior_t *p, const int64_t *h, int64_t *out) {
    int64_t Q = total_labels(p);
    int64_t maxlen = 0;
    for (int r = 0; r < p->R; ++r)
        if (p->Q[r] > maxlen) maxlen = p->Q[r];
    int64_t *fw = malloc(sizeof(int64_t) * maxlen), *bw = malloc(sizeof(int64_t) * maxlen);
    if (!fw || !bw) {
        free(fw);
        free(bw);
        return ORACLE_ERR_NOMEM;
    }
    int64_t cap = ipow(p->g, p->l1);
    int64_t hmin = INF64;
    for (int64_t q = 0; q < Q; ++q) {
        out[q] = h[q];
        if (h[q] < hmin) hmin = h[q];
    }
    for (int r = 0; r < p->R; ++r) {
        int64_t stride, nlines, len;
        axis_lines(p, r, &stride, &nlines, &len);
        for (int64_t l = 0; l < nlines; ++l) {
            int64_t *v = out + line_base(p, r, l);
            int64_t lmin = INF64;
            if (p->mode == PRIOR_PER_AXIS)
                for (int64_t i = 0; i < len; ++i)
                    if (v[i * stride] < lmin) lmin = v[i * stride];
            if (p->l1 == 1)
                lrms_line(v, len, stride, p->lambda, fw, bw);
            else
                grms_line(v, len, stride, p->lambda, p->g, p->l1, fw);
            if (p->mode == PRIOR_PER_AXIS) {
                /* per-axis truncation: min(|d|, g) on this axis alone */
                int64_t clip = lmin + (int64_t)p->lambda * cap;
                for (int64_t i = 0; i < len; ++i)
                    if (v[i * stride] > clip) v[i * stride] = clip;
            }
        }
    }
    if (p->mode == PRIOR_JOINT) {
        /* Eq. derivation1: clip by S_min + lambda f(g) */
        int64_t clip = hmin + (int64_t)p->lambda * cap;
        for (int64_t q = 0; q < Q; ++q)
            if (out[q] > clip) out[q] = clip;
    }
    free(fw);
    free(bw);
    return ORACLE_OK;
}

static int message(const oracle_prior_t *p, int tier, const int64_t *h, int64_t *out) {
    if (tier == 0) {
        message_brute(p, h, out);
        return ORACLE_OK;
    }
    return message_rms(p, h, out);
}

int oracle_message(const oracle_prior_t *p, int tier, const int64_t *h, int64_t *out) {
    int rc = check_prior(p);
    if (rc) return rc;
    return message(p, tier, h, out);
}

/* ------------------------------------------------------------------------ */
/* Scanline DP (Sec. 4.1): forward recurrence Eq. base with the boundary     */
/* condition Eq. DP_1D_2, then the backward recovery of the optimal path.    */
/* ------------------------------------------------------------------------ */

int oracle_scanline_dp(const int32_t *C, int W, int H, const oracle_prior_t *p, int tier,
                       int32_t *labels, int64_t *row_energy) {
    int rc = check_prior(p);
    if (rc) return rc;
    if (W < 1 || H < 1) return ORACLE_ERR_ARG;
    int64_t Q = total_labels(p);
    int64_t *S = malloc(sizeof(int64_t) * Q * W), *m = malloc(sizeof(int64_t) * Q);
    if (!S || !m) {
        free(S);
        free(m);
        return ORACLE_ERR_NOMEM;
    }
    for (int y = 0; y < H; ++y) {
        const int32_t *Cy = C + (int64_t)y * W * Q;
        /* x = 0: M(S(-1)) == 0 outside the image, so S(0) = C(0). */
        for (int64_t q = 0; q < Q; ++q) S[q] = Cy[q];
        for (int x = 1; x < W; ++x) {
            rc = message(p, tier, S + (int64_t)(x - 1) * Q, m);
            if (rc) goto out;
            for (int64_t q = 0; q < Q; ++q) {
                int64_t v = (int64_t)Cy[(int64_t)x * Q + q] + m[q];
                if (!fits32(m[q]) || !fits32(v)) {
                    rc = ORACLE_ERR_RANGE;
                    goto out;
                }
                S[(int64_t)x * Q + q] = v;
            }
        }
        /* minimum at the last column; lowest label index on ties */
        int64_t best = INF64, arg = 0;
        for (int64_t q = 0; q < Q; ++q)
            if (S[(int64_t)(W - 1) * Q + q] < best) {
                best = S[(int64_t)(W - 1) * Q + q];
                arg = q;
            }
        if (row_energy) row_energy[y] = best;
        labels[(int64_t)y * W + W - 1] = (int32_t)arg;
        /* backward recovery: v(x) = lowest argmin_q S(x, q) + V(q, v(x+1)) */
        for (int x = W - 2; x >= 0; --x) {
            int64_t next = labels[(int64_t)y * W + x + 1];
            int64_t bv = INF64, ba = 0;
            for (int64_t q = 0; q < Q; ++q) {
                int64_t v = S[(int64_t)x * Q + q] + oracle_prior(p, q, next);
                if (v < bv) {
                    bv = v;
                    ba = q;
                }
            }
            labels[(int64_t)y * W + x] = (int32_t)ba;
        }
    }
out:
    free(S);
    free(m);
    return rc;
}

/* Modified DP, Eq. DP_1D_3: S_Omega(x, v) = M(S_1(x-1)) + C(x, v) + M(S_-1(x+1))
 * with S_1 the forward and S_-1 the backward optimal sums of the row. */
int oracle_min_marginals(const int32_t *C, int W, int H, const oracle_prior_t *p, int tier,
                         int64_t *S_omega) {
    int rc = check_prior(p);
    if (rc) return rc;
    if (W < 1 || H < 1) return ORACLE_ERR_ARG;
    int64_t Q = total_labels(p);
    int64_t *F = malloc(sizeof(int64_t) * Q * W), *B = malloc(sizeof(int64_t) * Q * W);
    int64_t *m1 = malloc(sizeof(int64_t) * Q), *m2 = malloc(sizeof(int64_t) * Q);
    if (!F || !B || !m1 || !m2) {
        rc = ORACLE_ERR_NOMEM;
        goto out;
    }
    for (int y = 0; y < H; ++y) {
        const int32_t *Cy = C + (int64_t)y * W * Q;
        for (int64_t q = 0; q < Q; ++q) F[q] = Cy[q];
        for (int x = 1; x < W; ++x) {
            if ((rc = message(p, tier, F + (int64_t)(x - 1) * Q, m1))) goto out;
            for (int64_t q = 0; q < Q; ++q) F[(int64_t)x * Q + q] = Cy[(int64_t)x * Q + q] + m1[q];
        }
        for (int64_t q = 0; q < Q; ++q) B[(int64_t)(W - 1) * Q + q] = Cy[(int64_t)(W - 1) * Q + q];
        for (int x = W - 2; x >= 0; --x) {
            if ((rc = message(p, tier, B + (int64_t)(x + 1) * Q, m1))) goto out;
            for (int64_t q = 0; q < Q; ++q) B[(int64_t)x * Q + q] = Cy[(int64_t)x * Q + q] + m1[q];
        }
        for (int x = 0; x < W; ++x) {
            for (int64_t q = 0; q < Q; ++q) m1[q] = m2[q] = 0;
            if (x > 0 && (rc = message(p, tier, F + (int64_t)(x - 1) * Q, m1))) goto out;
            if (x < W - 1 && (rc = message(p, tier, B + (int64_t)(x + 1) * Q, m2))) goto out;
            for (int64_t q = 0; q < Q; ++q)
                S_omega[((int64_t)y * W + x) * Q + q] = m1[q] + Cy[(int64_t)x * Q + q] + m2[q];
        }
    }
out:
    free(F);
    free(B);
    free(m1);
    free(m2);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* EDP (Sec. 4.2, Algorithm 1).  Four directional sums S_k, k in            */
/* {+x, -x, +y, -y}, with x_k the neighbour behind x in direction k:        */
/*   x_{+x} = (x-1, y), x_{-x} = (x+1, y), x_{+y} = (x, y-1), x_{-y} = (x, y+1).*/
/* Message m_k(x, .) = M(floor(S_k(x_k, .) / 2)), or 0 when x_k is outside.  */
/* Update (Eq. DP_2D_base, data term added):                                */
/*   S_k'(x, .) = C(x, .) + sum_{k != -k'} m_k - m_{-k'}.                    */
/* Passes (P1..P4) each update two sums in place, in raster order.          */
/* Final (Eq. DP_2D_1 + C, Eq. DP_2D_2): S_Omega = C + sum_k m_k, argmin.   */
/* ------------------------------------------------------------------------ */

enum { KPX = 0, KMX = 1, KPY = 2, KMY = 3 };
static const int opposite[4] = {KMX, KPX, KMY, KPY};

typedef struct {
    int W, H;
    int64_t Q; /* labels per pixel (full space, or window size) */
} grid_t;

/* message into pixel (x, y) from direction k, computed from the current S_k */
typedef int (*msg_fn)(void *ctx, int k, int x, int y, int64_t *out);

typedef struct {
    const oracle_prior_t *p;
    int tier;
    grid_t g;
    int32_t *S; /* [4][H][W][Q] */
    int64_t *h;
    /* optional per-edge prior multipliers (locally adaptive lambda):
     * wh[y][x] for the edge (x, y)-(x+1, y), wv[y][x] for (x, y)-(x, y+1) */
    const uint8_t *wh, *wv;
} full_ctx;

static int neighbour(int k, int x, int y, int *xn, int *yn) {
    *xn = x;
    *yn = y;
    switch (k) {
    case KPX: *xn = x - 1; break;
    case KMX: *xn = x + 1; break;
    case KPY: *yn = y - 1; break;
    default: *yn = y + 1; break;
    }
    return 0;
}

static int full_msg(void *vctx, int k, int x, int y, int64_t *out) {
    full_ctx *c = vctx;
    int xn, yn;
    neighbour(k, x, y, &xn, &yn);
    if (xn < 0 || xn >= c->g.W || yn < 0 || yn >= c->g.H) {
        for (int64_t q = 0; q < c->g.Q; ++q) out[q] = 0;
        return ORACLE_OK;
    }
    const int32_t *s = c->S + (((int64_t)k * c->g.H + yn) * c->g.W + xn) * c->g.Q;
    for (int64_t q = 0; q < c->g.Q; ++q) c->h[q] = floor_half(s[q]);
    oracle_prior_t pe = *c->p;
    if (c->wh) {
        /* the prior of this edge: lambda times the edge's multiplier */
        const int w = (k == KPX || k == KMX) ? c->wh[(int64_t)y * c->g.W + (x < xn ? x : xn)]
                                             : c->wv[(int64_t)(y < yn ? y : yn) * c->g.W + x];
        pe.lambda = c->p->lambda * w;
    }
    int rc = message(&pe, c->tier, c->h, out);
    if (rc) return rc;
    for (int64_t q = 0; q < c->g.Q; ++q)
        if (!fits32(out[q])) return ORACLE_ERR_RANGE;
    return ORACLE_OK;
}

/* Shared driver of the four passes; `cost(x, y)` gives C at the pixel and
 * `msg` the four messages.  Labels are written as indexes into the pixel's
 * own label list (full space or window). */
static int edp_drive(grid_t g, int iters, const int32_t *C, int32_t *S, msg_fn msg, void *ctx,
                     int32_t *labels, int64_t *S_omega) {
    int64_t Q = g.Q;
    int64_t *m[4];
    for (int k = 0; k < 4; ++k) m[k] = malloc(sizeof(int64_t) * Q);
    int rc = ORACLE_OK;
    for (int k = 0; k < 4; ++k)
        if (!m[k]) rc = ORACLE_ERR_NOMEM;
    if (rc) goto out;
    /* initial sums: zero everywhere */
    memset(S, 0, sizeof(int32_t) * 4 * (size_t)g.H * g.W * Q);
    /* the sums each pass updates, in the order P1..P4 */
    static const int upd[4][2] = {{KPX, KPY}, {KMX, KPY}, {KPX, KMY}, {KMX, KMY}};
    static const int incx[4] = {1, 0, 1, 0}, incy[4] = {1, 1, 0, 0};
    for (int it = 0; it < iters; ++it)
        for (int pass = 0; pass < 4; ++pass)
            for (int yi = 0; yi < g.H; ++yi) {
                int y = incy[pass] ? yi : g.H - 1 - yi;
                for (int xi = 0; xi < g.W; ++xi) {
                    int x = incx[pass] ? xi : g.W - 1 - xi;
                    const int32_t *Cx = C + ((int64_t)y * g.W + x) * Q;
                    for (int k = 0; k < 4; ++k)
                        if ((rc = msg(ctx, k, x, y, m[k]))) goto out;
                    for (int u = 0; u < 2; ++u) {
                        int kp = upd[pass][u];
                        int32_t *dst = S + (((int64_t)kp * g.H + y) * g.W + x) * Q;
                        for (int64_t q = 0; q < Q; ++q) {
                            int64_t v = Cx[q];
                            for (int k = 0; k < 4; ++k) {
                                if (k == opposite[kp]) continue;
                                v += m[k][q];
                                if (!fits32(v)) {
                                    rc = ORACLE_ERR_RANGE;
                                    goto out;
                                }
                            }
                            v -= m[opposite[kp]][q];
                            if (!fits32(v)) {
                                rc = ORACLE_ERR_RANGE;
                                goto out;
                            }
                            dst[q] = (int32_t)v;
                        }
                    }
                }
            }
    /* marginal estimate and label decision */
    for (int y = 0; y < g.H; ++y)
        for (int x = 0; x < g.W; ++x) {
            const int32_t *Cx = C + ((int64_t)y * g.W + x) * Q;
            for (int k = 0; k < 4; ++k)
                if ((rc = msg(ctx, k, x, y, m[k]))) goto out;
            int64_t best = INF64, arg = 0;
            for (int64_t q = 0; q < Q; ++q) {
                int64_t v = Cx[q];
                for (int k = 0; k < 4; ++k) {
                    v += m[k][q];
                    if (!fits32(v)) {
                        rc = ORACLE_ERR_RANGE;
                        goto out;
                    }
                }
                if (S_omega) S_omega[((int64_t)y * g.W + x) * Q + q] = v;
                if (v < best) {
                    best = v;
                    arg = q;
                }
            }
            labels[(int64_t)y * g.W + x] = (int32_t)arg;
        }
out:
    for (int k = 0; k < 4; ++k) free(m[k]);
    return rc;
}

/* Full-label EDP.  S_out (optional) receives the final sums [4][H][W][Q]
 * (k order +x, -x, +y, -y); S_omega (optional) the marginal estimate. */
static int edp_full(const int32_t *C, int W, int H, const oracle_prior_t *p, int iters, int tier,
                    const uint8_t *wh, const uint8_t *wv, int32_t *labels, int32_t *S_out, int64_t *S_omega) {
    int rc = check_prior(p);
    if (rc) return rc;
    if (W < 1 || H < 1 || iters < 0) return ORACLE_ERR_ARG;
    if ((wh == NULL) != (wv == NULL)) return ORACLE_ERR_ARG;
    full_ctx c;
    c.p = p;
    c.wh = wh;
    c.wv = wv;
    c.tier = tier;
    c.g.W = W;
    c.g.H = H;
    c.g.Q = total_labels(p);
    int32_t *S = S_out ? S_out : malloc(sizeof(int32_t) * 4 * (size_t)W * H * c.g.Q);
    c.S = S;
    c.h = malloc(sizeof(int64_t) * c.g.Q);
    if (!S || !c.h) {
        if (!S_out) free(S);
        free(c.h);
        return ORACLE_ERR_NOMEM;
    }
    rc = edp_drive(c.g, iters, C, S, full_msg, &c, labels, S_omega);
    if (!S_out) free(S);
    free(c.h);
    return rc;
}

int oracle_edp(const int32_t *C, int W, int H, const oracle_prior_t *p, int iters, int tier,
               int32_t *labels, int32_t *S_out, int64_t *S_omega) {
    return edp_full(C, W, H, p, iters, tier, NULL, NULL, labels, S_out, S_omega);
}

/* EDP with a locally adaptive prior (the text below Eq. Smooth_value_t):
 * the prior of every grid edge is lambda times the edge's multiplier,
 * wh[y][x] for (x, y)-(x+1, y) and wv[y][x] for (x, y)-(x, y+1) (uint8,
 * [H][W]; the last column of wh and the last row of wv are not read). */
int oracle_edp_weighted(const int32_t *C, int W, int H, const oracle_prior_t *p, int iters, int tier,
                        const uint8_t *wh, const uint8_t *wv, int32_t *labels) {
    if (!wh || !wv) return ORACLE_ERR_ARG;
    return edp_full(C, W, H, p, iters, tier, wh, wv, labels, NULL, NULL);
}

/* The paper's adaptive rule, read as per-edge multipliers: an edge whose
 * intensity step |I(x') - I(x)| is below `thresh` gets `factor` (the paper:
 * 2 lambda where the local gradient of I_t is below 10), every other edge 1.
 * Entries without an edge (last column of wh, last row of wv) are 1. */
int oracle_edge_weights(const uint8_t *I, int W, int H, int pitch, int thresh, int factor, uint8_t *wh,
                        uint8_t *wv) {
    if (!I || !wh || !wv || W < 1 || H < 1 || pitch < W || factor < 0 || factor > 255) return ORACLE_ERR_ARG;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int v = I[(int64_t)y * pitch + x];
            int h = 1, u = 1;
            if (x + 1 < W) {
                const int d = I[(int64_t)y * pitch + x + 1] - v;
                h = (d < 0 ? -d : d) < thresh ? factor : 1;
            }
            if (y + 1 < H) {
                const int d = I[(int64_t)(y + 1) * pitch + x] - v;
                u = (d < 0 ? -d : d) < thresh ? factor : 1;
            }
            wh[(int64_t)y * W + x] = (uint8_t)h;
            wv[(int64_t)y * W + x] = (uint8_t)u;
        }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Windowed EDP: every pixel keeps its own box of win^R labels (centre from  */
/* a proposal).  A message from x_k to x is the plain min-convolution        */
/*   m(v) = min_{u in box(x_k)} floor(S(x_k, u)/2) + V(u, v),  v in box(x)   */
/* evaluated by brute force over the two boxes.                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    const oracle_prior_t *p;
    grid_t g;
    int win;
    int32_t *S;
    const int32_t *centre;
    int64_t *h;
} win_ctx;

static int64_t box_label(const oracle_prior_t *p, const int64_t lo[3], int win, int64_t w) {
    int64_t c0 = lo[0] + w % win;
    if (p->R == 1) return c0;
    return c0 + p->Q[0] * (lo[1] + w / win);
}

static int win_msg(void *vctx, int k, int x, int y, int64_t *out) {
    win_ctx *c = vctx;
    int xn, yn;
    neighbour(k, x, y, &xn, &yn);
    if (xn < 0 || xn >= c->g.W || yn < 0 || yn >= c->g.H) {
        for (int64_t q = 0; q < c->g.Q; ++q) out[q] = 0;
        return ORACLE_OK;
    }
    int64_t lo_src[3], lo_dst[3];
    clamp_centre(c->p, c->win, c->centre + ((int64_t)yn * c->g.W + xn) * c->p->R, lo_src);
    clamp_centre(c->p, c->win, c->centre + ((int64_t)y * c->g.W + x) * c->p->R, lo_dst);
    const int32_t *s = c->S + (((int64_t)k * c->g.H + yn) * c->g.W + xn) * c->g.Q;
    for (int64_t v = 0; v < c->g.Q; ++v) {
        int64_t qv = box_label(c->p, lo_dst, c->win, v);
        int64_t best = INF64;
        for (int64_t u = 0; u < c->g.Q; ++u) {
            int64_t qu = box_label(c->p, lo_src, c->win, u);
            int64_t t = floor_half(s[u]) + oracle_prior(c->p, qu, qv);
            if (t < best) best = t;
        }
        if (!fits32(best)) return ORACLE_ERR_RANGE;
        out[v] = best;
    }
    return ORACLE_OK;
}

/* labels receive full-space linear label indexes.  S_out (optional)
 * receives the final sums [4][H][W][win^R] in box coordinates (k order +x,
 * -x, +y, -y). */
int oracle_edp_windowed(const int32_t *Cw, const int32_t *centre, int W, int H,
                        const oracle_prior_t *p, int win, int iters, int32_t *labels, int32_t *S_out) {
    int rc = check_prior(p);
    if (rc) return rc;
    if (W < 1 || H < 1 || iters < 0 || p->R > 2 || win < 1 || (win & 1) == 0)
        return ORACLE_ERR_ARG;
    for (int r = 0; r < p->R; ++r)
        if (p->Q[r] < win) return ORACLE_ERR_ARG;
    win_ctx c;
    c.p = p;
    c.win = win;
    c.centre = centre;
    c.g.W = W;
    c.g.H = H;
    c.g.Q = p->R == 1 ? win : (int64_t)win * win;
    c.S = S_out ? S_out : malloc(sizeof(int32_t) * 4 * (size_t)W * H * c.g.Q);
    if (!c.S) return ORACLE_ERR_NOMEM;
    rc = edp_drive(c.g, iters, Cw, c.S, win_msg, &c, labels, NULL);
    if (!rc)
        for (int64_t i = 0; i < (int64_t)W * H; ++i) {
            int64_t lo[3];
            clamp_centre(p, win, centre + i * p->R, lo);
            labels[i] = (int32_t)box_label(p, lo, win, labels[i]);
        }
    if (!S_out) free(c.S);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Energy, Eq. GE_objective_function on the 4-connected grid:               */
/* data term + right-neighbour edges + down-neighbour edges.                */
/* ------------------------------------------------------------------------ */

static int energy_full(const int32_t *C, const int32_t *labels, int W, int H, const oracle_prior_t *p,
                       const uint8_t *wh, const uint8_t *wv, int64_t *out4) {
    int rc = check_prior(p);
    if (rc) return rc;
    int64_t Q = total_labels(p);
    int64_t data = 0, sh = 0, sv = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t l = labels[(int64_t)y * W + x];
            if (l < 0 || l >= Q) return ORACLE_ERR_ARG;
            if (C) data += C[((int64_t)y * W + x) * Q + l];
            const int64_t i = (int64_t)y * W + x;
            if (x + 1 < W) sh += (wh ? wh[i] : 1) * oracle_prior(p, l, labels[i + 1]);
            if (y + 1 < H) sv += (wv ? wv[i] : 1) * oracle_prior(p, l, labels[i + W]);
        }
    out4[0] = data;
    out4[1] = sh;
    out4[2] = sv;
    out4[3] = data + sh + sv;
    return ORACLE_OK;
}

int oracle_energy(const int32_t *C, const int32_t *labels, int W, int H, const oracle_prior_t *p,
                  int64_t *out4) {
    return energy_full(C, labels, W, H, p, NULL, NULL, out4);
}

/* Eq. GE_objective_function with per-edge multipliers of the prior (see
 * oracle_edp_weighted). */
int oracle_energy_weighted(const int32_t *C, const int32_t *labels, int W, int H, const oracle_prior_t *p,
                           const uint8_t *wh, const uint8_t *wv, int64_t *out4) {
    if (!wh || !wv) return ORACLE_ERR_ARG;
    return energy_full(C, labels, W, H, p, wh, wv, out4);
}
