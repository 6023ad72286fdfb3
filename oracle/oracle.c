/*
 * CPU oracle for the band-FHT + bend-limited DP method of
 * "A Method of Detecting End-To-End Curves of Limited Curvature"
 * (Panfilova, Aliev, Kunina, Postnikov, Nikolaev; arXiv 1912.01884).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA library against a plain,
 * slow, obviously correct restatement of the method.  It shares no code,
 * header, table or constant with the CUDA sources.
 *
 * Everything is plain loops in double precision (exact for every integer
 * image the library accepts), plus float32 copies of the FHT recursion, of
 * the DP and of the queries (smoothing and bend angle, through-point, padded
 * vertices, two polylines): the float path of the library takes its argmax
 * decisions in float32, so the oracle takes the same decisions in the same
 * precision.
 *
 * Conventions (the paper is silent or garbled on each; the readings are the
 * ones listed with the design notes):
 *   n = h/k rows per band, a power of two; W = w + n (Sec. 2.1: each band is
 *   extended to the right by h/k zero columns).
 *   A link of band i runs from column x_i on the band's first row to column
 *   x_i + d on its last row, |d| <= n-1 (45 degrees, Sec. 2 def. 2).  The
 *   paper's "shift" is n - d (Eq. 1, Eq. 2); the oracle uses d directly.
 *   Dyadic pattern off_s(y) of a line of shift s >= 0 over m rows:
 *     m == 1: off_0(0) = 0
 *     else:   first m/2 rows follow off_{s>>1} over m/2 rows, the last m/2
 *             rows follow ceil(s/2) + off_{s>>1} over m/2 rows.
 *   Hough images (Sec. 2.1), cyclic over the padded width W:
 *     H+(x, s) = sum_y P(y, (x + off_s(y)) mod W)
 *     H-(x, s) = sum_y P(y, (x - off_s(y)) mod W)
 *   and H(x, d) = H+(x, d) for d >= 0, H-(x, -d) for d < 0.
 *   Hough array layout: H[band][sign][s][x], sign 0 = "+", 1 = "-",
 *   s in [0, n), x in [0, W).
 *   Value array layout: V[band][d + n - 1][x], x in [0, w).
 *   Dead states (no admissible continuation) hold -infinity.
 *   Ties resolve to the lexicographically smallest (x_0, d_0, ..., d_{k-1})
 *   with d ordered numerically.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NEG (-INFINITY)

/* ---------------------------------------------------------------------------
 * Sec. 2.1 (FHT of each band, refs [10], [34]): the dyadic line pattern.
 * off(m, s, y) is the column offset, on row y, of the line of shift s over m
 * rows.  Written straight from the recursive definition above.
 * ------------------------------------------------------------------------ */
static int off_rec(int m, int s, int y) {
    if (m == 1) return 0;
    int half = m / 2;
    int s_half = s >> 1;
    if (y < half) return off_rec(half, s_half, y);
    return (s - s_half) + off_rec(half, s_half, y - half);
}

/* off[s * n + y] = off_s(y) for s, y in [0, n).  Returns 0, or -1 when n is
 * not a power of two. */
int oracle_off_table(int n, int32_t *off) {
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    for (int s = 0; s < n; ++s)
        for (int y = 0; y < n; ++y) off[(size_t)s * n + y] = off_rec(n, s, y);
    return 0;
}

/* Pixel of band b, row y, padded column c in [0, W): zero in the padding. */
static double band_pixel(const double *img, int w, int n, int b, int y, int c) {
    if (c >= w) return 0.0;
    return img[((size_t)b * n + y) * w + c];
}

static int mod_w(long v, int W) {
    long r = v % W;
    return (int)(r < 0 ? r + W : r);
}

/* ---------------------------------------------------------------------------
 * Sec. 2.1: the Hough images H_0..H_{k-1} by DIRECT summation along every
 * dyadic line of every zero-padded band (the definition itself, O(n^2 W)).
 * img: h x w row-major doubles.  H: [k][2][n][W].
 * ------------------------------------------------------------------------ */
int oracle_fht_direct_f64(const double *img, int h, int w, int k, double *H) {
    if (k < 1 || h % k != 0) return -1;
    int n = h / k;
    if ((n & (n - 1)) != 0) return -1;
    int W = w + n;
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * n);
    if (!off) return -2;
    oracle_off_table(n, off);
    for (int b = 0; b < k; ++b)
        for (int sign = 0; sign < 2; ++sign)
            for (int s = 0; s < n; ++s)
                for (int x = 0; x < W; ++x) {
                    double acc = 0.0;
                    for (int y = 0; y < n; ++y) {
                        long o = off[(size_t)s * n + y];
                        int c = mod_w(sign == 0 ? x + o : x - o, W);
                        acc += band_pixel(img, w, n, b, y, c);
                    }
                    H[(((size_t)b * 2 + sign) * n + s) * W + x] = acc;
                }
    free(off);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Sec. 2.1 (FHT, refs [10], [34]): the same Hough images by the dyadic
 * recursion.  A sub-band of m rows is the union of its top half (A) and its
 * bottom half (B); its line of shift s is A's line of shift s>>1 followed by
 * B's line of shift s>>1 moved ceil(s/2) columns (right for "+", left for
 * "-").  So out(x, s) = A(x, s>>1) + B(x +/- ceil(s/2), s>>1), cyclic in W.
 * In float32 this fixes the summation tree: every value is (top half) +
 * (bottom half), recursively, which is the order the CUDA path must follow.
 * ------------------------------------------------------------------------ */
#define ORACLE_DEFINE_FHT_RECURSIVE(T, SUFFIX)                                   \
    /* out: [m][W] for the rows [y0, y0 + m) of band b, one sign. */             \
    static void fht_rec_##SUFFIX(const T *img, int w, int n, int W, int b,       \
                                 int sign, int y0, int m, T *out) {              \
        if (m == 1) {                                                            \
            for (int x = 0; x < W; ++x)                                          \
                out[x] = (x < w) ? img[((size_t)b * n + y0) * w + x] : (T)0;     \
            return;                                                              \
        }                                                                        \
        int half = m / 2;                                                        \
        T *top = (T *)malloc(sizeof(T) * (size_t)half * W);                      \
        T *bot = (T *)malloc(sizeof(T) * (size_t)half * W);                      \
        fht_rec_##SUFFIX(img, w, n, W, b, sign, y0, half, top);                  \
        fht_rec_##SUFFIX(img, w, n, W, b, sign, y0 + half, half, bot);           \
        for (int s = 0; s < m; ++s) {                                            \
            int s_half = s >> 1;                                                 \
            int move = s - s_half;                                               \
            for (int x = 0; x < W; ++x) {                                        \
                int xb = mod_w(sign == 0 ? (long)x + move : (long)x - move, W);  \
                out[(size_t)s * W + x] =                                         \
                    top[(size_t)s_half * W + x] + bot[(size_t)s_half * W + xb];  \
            }                                                                    \
        }                                                                        \
        free(top);                                                               \
        free(bot);                                                               \
    }                                                                            \
    int oracle_fht_recursive_##SUFFIX(const T *img, int h, int w, int k, T *H) { \
        if (k < 1 || h % k != 0) return -1;                                      \
        int n = h / k;                                                           \
        if ((n & (n - 1)) != 0) return -1;                                       \
        int W = w + n;                                                           \
        for (int b = 0; b < k; ++b)                                              \
            for (int sign = 0; sign < 2; ++sign)                                 \
                fht_rec_##SUFFIX(img, w, n, W, b, sign, 0, n,                    \
                                 H + ((size_t)b * 2 + sign) * n * W);            \
        return 0;                                                                \
    }

ORACLE_DEFINE_FHT_RECURSIVE(double, f64)
ORACLE_DEFINE_FHT_RECURSIVE(float, f32)

/* ---------------------------------------------------------------------------
 * Sec. 2.2-2.3 (Eqs. 3-4, RangeMaxQ): the bottom-up max-plus DP over the
 * bands, with the bend restriction |d_{i+1} - d_i| <= B (the integer form of
 * the bend window; B >= 2n-2 is the unrestricted Subproblem 2).
 *   V_{k-1}(x, d) = H_{k-1}(x, d)                  if x + d in [0, w)
 *   V_i(x, d)     = H_i(x, d) + max_{|e-d|<=B} V_{i+1}(x + d, e)
 *                                                  if x + d in [0, w)
 *   dead otherwise (and dead when every e in the window is dead).
 * The window maximum is a plain scan over the window (no range-max
 * structure: the structure only changes the cost, not the result).
 * H: [k][2][n][W], V: [k][2n-1][w].
 * ------------------------------------------------------------------------ */
/* win (optional, NULL = none): [k][2] allowed displacements [lo_i, hi_i] of
 * each band; links outside are dead.  This restriction is the pruned DP of
 * the learned window proposal, which is not part of the paper. */
#define ORACLE_DEFINE_DP(T, SUFFIX)                                              \
    static T hough_at_##SUFFIX(const T *H, int n, int W, int b, int x, int d) {  \
        int sign = d >= 0 ? 0 : 1;                                               \
        int s = d >= 0 ? d : -d;                                                 \
        return H[(((size_t)b * 2 + sign) * n + s) * W + x];                      \
    }                                                                            \
    int oracle_dp_win_##SUFFIX(const T *H, int h, int w, int k, int B,           \
                               const int32_t *win, T *V) {                       \
        if (k < 1 || h % k != 0 || B < 0) return -1;                             \
        int n = h / k;                                                           \
        int W = w + n;                                                           \
        int D = 2 * n - 1;                                                       \
        for (int b = k - 1; b >= 0; --b)                                         \
            for (int d = -(n - 1); d <= n - 1; ++d)                              \
                for (int x = 0; x < w; ++x) {                                    \
                    T *out = &V[((size_t)b * D + (d + n - 1)) * w + x];          \
                    int xn = x + d;                                              \
                    int outside = win && (d < win[2 * b] || d > win[2 * b + 1]); \
                    if (xn < 0 || xn >= w || outside) {                          \
                        *out = (T)ORACLE_NEG;                                    \
                        continue;                                                \
                    }                                                            \
                    T hv = hough_at_##SUFFIX(H, n, W, b, x, d);                  \
                    if (b == k - 1) {                                            \
                        *out = hv;                                               \
                        continue;                                                \
                    }                                                            \
                    T best = (T)ORACLE_NEG;                                      \
                    for (int e = d - B; e <= d + B; ++e) {                       \
                        if (e < -(n - 1) || e > n - 1) continue;                 \
                        T v = V[((size_t)(b + 1) * D + (e + n - 1)) * w + xn];   \
                        if (v > best) best = v;                                  \
                    }                                                            \
                    *out = (best == (T)ORACLE_NEG) ? (T)ORACLE_NEG : hv + best;  \
                }                                                                \
        return 0;                                                                \
    }                                                                            \
    int oracle_dp_##SUFFIX(const T *H, int h, int w, int k, int B, T *V) {       \
        return oracle_dp_win_##SUFFIX(H, h, w, k, B, NULL, V);                   \
    }

ORACLE_DEFINE_DP(double, f64)
ORACLE_DEFINE_DP(float, f32)

/* ---------------------------------------------------------------------------
 * Sec. 2.2 Eq. 5 and the main problem (steps 2-3): pick the best top point
 * and read the polyline back band by band.
 *   (x_0, d_0) = lexicographically smallest argmax of V_0 over x, d.
 *   x_{i+1} = x_i + d_i (Eq. 2 / Eq. 5 with shift = n - d).
 *   d_{i+1} = smallest e with |e - d_i| <= B maximising V_{i+1}(x_{i+1}, e).
 * Because V_{i+1}(x, e) is the exact best continuation, this greedy choice
 * yields the lexicographically smallest optimal polyline.
 * x: k+1 vertices, d: k displacements.  Returns the optimal score.
 * ------------------------------------------------------------------------ */
#define ORACLE_DEFINE_BACKTRACK(T, SUFFIX)                                       \
    double oracle_backtrack_##SUFFIX(const T *V, int h, int w, int k, int B,     \
                                     int32_t *xs, int32_t *ds) {                 \
        int n = h / k;                                                           \
        int D = 2 * n - 1;                                                       \
        T best = (T)ORACLE_NEG;                                                  \
        int bx = 0, bd = 0;                                                      \
        for (int x = 0; x < w; ++x)                                              \
            for (int d = -(n - 1); d <= n - 1; ++d) {                            \
                T v = V[((size_t)0 * D + (d + n - 1)) * w + x];                  \
                if (v > best) {                                                  \
                    best = v;                                                    \
                    bx = x;                                                      \
                    bd = d;                                                      \
                }                                                                \
            }                                                                    \
        if (best == (T)ORACLE_NEG) { /* no admissible polyline */               \
            for (int i = 0; i <= k; ++i) xs[i] = -1;                             \
            for (int i = 0; i < k; ++i) ds[i] = 0;                               \
            return (double)ORACLE_NEG;                                           \
        }                                                                        \
        xs[0] = bx;                                                              \
        ds[0] = bd;                                                              \
        for (int i = 1; i < k; ++i) {                                            \
            int xi = xs[i - 1] + ds[i - 1];                                      \
            xs[i] = xi;                                                          \
            T bv = (T)ORACLE_NEG;                                                \
            int be = 0;                                                          \
            for (int e = ds[i - 1] - B; e <= ds[i - 1] + B; ++e) {               \
                if (e < -(n - 1) || e > n - 1) continue;                         \
                T v = V[((size_t)i * D + (e + n - 1)) * w + xi];                 \
                if (v > bv) {                                                    \
                    bv = v;                                                      \
                    be = e;                                                      \
                }                                                                \
            }                                                                    \
            ds[i] = be;                                                          \
        }                                                                        \
        xs[k] = xs[k - 1] + ds[k - 1];                                           \
        return (double)best;                                                     \
    }

ORACLE_DEFINE_BACKTRACK(double, f64)
ORACLE_DEFINE_BACKTRACK(float, f32)

/* ---------------------------------------------------------------------------
 * Sec. 2.1 (the query of Subproblem 1) by the plain definition: the sum of
 * the pixels along the polyline, link by link, row by row (double).
 * Returns -infinity if a vertex leaves [0, w) or |d_i| > n-1.
 * ------------------------------------------------------------------------ */
double oracle_path_score_f64(const double *img, int h, int w, int k, int x0,
                             const int32_t *ds) {
    int n = h / k;
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * n);
    if (!off) return ORACLE_NEG;
    oracle_off_table(n, off);
    double acc = 0.0;
    int x = x0;
    if (x < 0 || x >= w) acc = ORACLE_NEG;
    for (int i = 0; i < k && acc != ORACLE_NEG; ++i) {
        int d = ds[i];
        int s = d >= 0 ? d : -d;
        if (s > n - 1 || x + d < 0 || x + d >= w) {
            acc = ORACLE_NEG;
            break;
        }
        for (int y = 0; y < n; ++y) {
            int c = x + (d >= 0 ? 1 : -1) * off[(size_t)s * n + y];
            acc += img[((size_t)i * n + y) * w + c];
        }
        x += d;
    }
    free(off);
    return acc;
}

/* ---------------------------------------------------------------------------
 * Brute force over every admissible polyline (tiny images only): x_0 in
 * [0, w), each d_i in [-(n-1), n-1], vertices in [0, w), |d_{i+1}-d_i| <= B.
 * Enumerated in lexicographic order; the first strictly better score wins, so
 * the result is the lexicographically smallest optimum.  The score of each
 * candidate is recomputed from scratch by oracle_path_score_f64.
 * ------------------------------------------------------------------------ */
typedef struct {
    const double *img;
    const int32_t *win;
    int h, w, k, n, B;
    int32_t *cur_d;
    int cur_x0;
    double best;
    int32_t *best_x;
    int32_t *best_d;
    long visited;
} brute_state;

static void brute_rec(brute_state *st, int i, int x) {
    int n = st->n;
    for (int d = -(n - 1); d <= n - 1; ++d) {
        if (i > 0) {
            int prev = st->cur_d[i - 1];
            if (d < prev - st->B || d > prev + st->B) continue;
        }
        if (x + d < 0 || x + d >= st->w) continue;
        if (st->win && (d < st->win[2 * i] || d > st->win[2 * i + 1])) continue;
        st->cur_d[i] = d;
        if (i + 1 < st->k) {
            brute_rec(st, i + 1, x + d);
        } else {
            st->visited++;
            double sc = oracle_path_score_f64(st->img, st->h, st->w, st->k,
                                              st->cur_x0, st->cur_d);
            if (sc > st->best) {
                st->best = sc;
                int xx = st->cur_x0;
                for (int j = 0; j < st->k; ++j) {
                    st->best_x[j] = xx;
                    st->best_d[j] = st->cur_d[j];
                    xx += st->cur_d[j];
                }
                st->best_x[st->k] = xx;
            }
        }
    }
}

double oracle_brute_win_f64(const double *img, int h, int w, int k, int B,
                            const int32_t *win, int32_t *xs, int32_t *ds, long *visited) {
    brute_state st;
    st.img = img;
    st.win = win;
    st.h = h;
    st.w = w;
    st.k = k;
    st.n = h / k;
    st.B = B;
    st.cur_d = (int32_t *)calloc((size_t)k, sizeof(int32_t));
    st.best = ORACLE_NEG;
    st.best_x = xs;
    st.best_d = ds;
    st.visited = 0;
    for (int x0 = 0; x0 < w; ++x0) {
        st.cur_x0 = x0;
        brute_rec(&st, 0, x0);
    }
    free(st.cur_d);
    if (visited) *visited = st.visited;
    if (st.best == ORACLE_NEG) {
        for (int i = 0; i <= k; ++i) xs[i] = -1;
        for (int i = 0; i < k; ++i) ds[i] = 0;
    }
    return st.best;
}

double oracle_brute_f64(const double *img, int h, int w, int k, int B,
                        int32_t *xs, int32_t *ds, long *visited) {
    return oracle_brute_win_f64(img, h, w, k, B, NULL, xs, ds, visited);
}

/* ---------------------------------------------------------------------------
 * The whole method (FHT recursion, DP, backtrack) in double: the CPU
 * baseline.  Scratch is allocated here; returns the optimal score.
 * ------------------------------------------------------------------------ */
double oracle_detect_f64(const double *img, int h, int w, int k, int B,
                         int32_t *xs, int32_t *ds) {
    int n = h / k;
    int W = w + n;
    double *H = (double *)malloc(sizeof(double) * (size_t)k * 2 * n * W);
    double *V = (double *)malloc(sizeof(double) * (size_t)k * (2 * n - 1) * w);
    if (!H || !V) {
        free(H);
        free(V);
        return NAN;
    }
    oracle_fht_recursive_f64(img, h, w, k, H);
    oracle_dp_f64(H, h, w, k, B, V);
    double s = oracle_backtrack_f64(V, h, w, k, B, xs, ds);
    free(H);
    free(V);
    return s;
}

/* The method restricted to per-band displacement windows (win [k][2]). */
double oracle_detect_win_f64(const double *img, int h, int w, int k, int B,
                             const int32_t *win, int32_t *xs, int32_t *ds) {
    int n = h / k;
    int W = w + n;
    double *H = (double *)malloc(sizeof(double) * (size_t)k * 2 * n * W);
    double *V = (double *)malloc(sizeof(double) * (size_t)k * (2 * n - 1) * w);
    if (!H || !V) {
        free(H);
        free(V);
        return NAN;
    }
    oracle_fht_recursive_f64(img, h, w, k, H);
    oracle_dp_win_f64(H, h, w, k, B, win, V);
    double s = oracle_backtrack_f64(V, h, w, k, B, xs, ds);
    free(H);
    free(V);
    return s;
}

/* The same in float32: the decisions the float path of the library takes. */
double oracle_detect_f32(const float *img, int h, int w, int k, int B,
                         int32_t *xs, int32_t *ds) {
    int n = h / k;
    int W = w + n;
    float *H = (float *)malloc(sizeof(float) * (size_t)k * 2 * n * W);
    float *V = (float *)malloc(sizeof(float) * (size_t)k * (2 * n - 1) * w);
    if (!H || !V) {
        free(H);
        free(V);
        return NAN;
    }
    oracle_fht_recursive_f32(img, h, w, k, H);
    oracle_dp_f32(H, h, w, k, B, V);
    double s = oracle_backtrack_f32(V, h, w, k, B, xs, ds);
    free(H);
    free(V);
    return s;
}

/* ---------------------------------------------------------------------------
 * The main problem (Sec. 2.3: the Welsh M-estimate of the polyline).
 *
 * Step 1: every row convolved with a one-dimensional Gaussian.  Reading: the
 * discrete Gaussian of half-width r, i.e. the binomial weights C(2r, r + t),
 * t in [-r, r], unnormalised (the common factor 4^r scales every polyline
 * sum alike and leaves the argmax unchanged); zero outside [0, w).  A uint8
 * image then gives exact integers.
 *   out(y, x) = sum_t C(2r, r + t) * img(y, x + t)
 * ------------------------------------------------------------------------ */
static double binom(int a, int b) {
    double c = 1.0;
    for (int i = 1; i <= b; ++i) c = c * (a - b + i) / i;
    return c;
}

int oracle_gauss_rows_f64(const double *img, int h, int w, int r, double *out) {
    if (r < 0) return -1;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double acc = 0.0;
            for (int t = -r; t <= r; ++t) {
                int c = x + t;
                if (c < 0 || c >= w) continue;
                acc += binom(2 * r, r + t) * img[(size_t)y * w + c];
            }
            out[(size_t)y * w + x] = acc;
        }
    return 0;
}

/* Step 2's bending-angle restriction (Sec. 2.3, Fig. 5).  A link of
 * displacement d over a band of n rows has inclination atan(d / n) from the
 * vertical (the paper's shift = h + h tg(phi) with h the band height, so
 * d = n tg(phi)); the bend angle between consecutive links d, e is
 * |atan(e / n) - atan(d / n)|, and e is admissible after d when that is at
 * most gamma.  Every |e| <= n - 1 already has its inclination inside
 * [-pi/4, pi/4], the second condition of Eqs. 6-7.  This is the plain
 * definition, evaluated in double pair by pair; since atan is increasing the
 * admissible e form one interval (the union of the ranges of Eqs. 6 and 7),
 * stored as lohi: [2n-1][2], entry d + n - 1 = {lo(d), hi(d)}. */
int oracle_angle_window(int n, double gamma, int32_t *lohi) {
    if (n < 1 || !(gamma >= 0.0)) return -1;
    for (int d = -(n - 1); d <= n - 1; ++d) {
        int lo = n, hi = -n;
        for (int e = -(n - 1); e <= n - 1; ++e) {
            double bend = fabs(atan((double)e / n) - atan((double)d / n));
            if (bend <= gamma) {
                if (e < lo) lo = e;
                if (e > hi) hi = e;
            }
        }
        lohi[2 * (d + n - 1)] = lo;
        lohi[2 * (d + n - 1) + 1] = hi;
    }
    return 0;
}

/* The DP of Sec. 2.3 (the RangeMaxQ steps): as oracle_dp_f64, with the
 * continuation window of displacement d being [lo(d), hi(d)] from lohi
 * instead of [d - B, d + B]; the window maximum is a plain scan. */
int oracle_dp_angle_f64(const double *H, int h, int w, int k, const int32_t *lohi,
                        double *V) {
    if (k < 1 || h % k != 0) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    for (int b = k - 1; b >= 0; --b)
        for (int d = -(n - 1); d <= n - 1; ++d)
            for (int x = 0; x < w; ++x) {
                double *out = &V[((size_t)b * D + (d + n - 1)) * w + x];
                int xn = x + d;
                if (xn < 0 || xn >= w) {
                    *out = ORACLE_NEG;
                    continue;
                }
                double hv = hough_at_f64(H, n, W, b, x, d);
                if (b == k - 1) {
                    *out = hv;
                    continue;
                }
                double best = ORACLE_NEG;
                for (int e = lohi[2 * (d + n - 1)]; e <= lohi[2 * (d + n - 1) + 1]; ++e) {
                    double v = V[((size_t)(b + 1) * D + (e + n - 1)) * w + xn];
                    if (v > best) best = v;
                }
                *out = (best == ORACLE_NEG) ? ORACLE_NEG : hv + best;
            }
    return 0;
}

/* Step 3 and the read-back (Eq. 5) with the angle windows: the
 * lexicographically smallest argmax of V_0, then band by band the smallest
 * e in [lo(d_{i-1}), hi(d_{i-1})] maximising V_i(x_i, e). */
double oracle_backtrack_angle_f64(const double *V, int h, int w, int k, const int32_t *lohi,
                                  int32_t *xs, int32_t *ds) {
    int n = h / k;
    int D = 2 * n - 1;
    double best = ORACLE_NEG;
    int bx = 0, bd = 0;
    for (int x = 0; x < w; ++x)
        for (int d = -(n - 1); d <= n - 1; ++d) {
            double v = V[(size_t)(d + n - 1) * w + x];
            if (v > best) {
                best = v;
                bx = x;
                bd = d;
            }
        }
    if (best == ORACLE_NEG) {
        for (int i = 0; i <= k; ++i) xs[i] = -1;
        for (int i = 0; i < k; ++i) ds[i] = 0;
        return ORACLE_NEG;
    }
    xs[0] = bx;
    ds[0] = bd;
    for (int i = 1; i < k; ++i) {
        int xi = xs[i - 1] + ds[i - 1];
        xs[i] = xi;
        int p = ds[i - 1] + n - 1;
        double bv = ORACLE_NEG;
        int be = lohi[2 * p];
        for (int e = lohi[2 * p]; e <= lohi[2 * p + 1]; ++e) {
            double v = V[((size_t)i * D + (e + n - 1)) * w + xi];
            if (v > bv) {
                bv = v;
                be = e;
            }
        }
        ds[i] = be;
    }
    xs[k] = xs[k - 1] + ds[k - 1];
    return best;
}

/* Brute force over every polyline whose consecutive links satisfy the bend
 * angle restriction tested directly, |atan(d_{i+1}/n) - atan(d_i/n)| <=
 * gamma (no window table), vertices in [0, w); lexicographic enumeration,
 * first strict maximum kept.  Tiny images only. */
typedef struct {
    const double *img;
    int h, w, k, n;
    double gamma;
    int32_t *cur_d;
    int cur_x0;
    double best;
    int32_t *best_x;
    int32_t *best_d;
    long visited;
} brute_angle_state;

static void brute_angle_rec(brute_angle_state *st, int i, int x) {
    int n = st->n;
    for (int d = -(n - 1); d <= n - 1; ++d) {
        if (i > 0) {
            double diff = atan((double)d / n) - atan((double)st->cur_d[i - 1] / n);
            if (fabs(diff) > st->gamma) continue;
        }
        if (x + d < 0 || x + d >= st->w) continue;
        st->cur_d[i] = d;
        if (i + 1 < st->k) {
            brute_angle_rec(st, i + 1, x + d);
        } else {
            st->visited++;
            double sc = oracle_path_score_f64(st->img, st->h, st->w, st->k, st->cur_x0,
                                              st->cur_d);
            if (sc > st->best) {
                st->best = sc;
                int xx = st->cur_x0;
                for (int j = 0; j < st->k; ++j) {
                    st->best_x[j] = xx;
                    st->best_d[j] = st->cur_d[j];
                    xx += st->cur_d[j];
                }
                st->best_x[st->k] = xx;
            }
        }
    }
}

double oracle_brute_angle_f64(const double *img, int h, int w, int k, double gamma,
                              int32_t *xs, int32_t *ds, long *visited) {
    brute_angle_state st;
    st.img = img;
    st.h = h;
    st.w = w;
    st.k = k;
    st.n = h / k;
    st.gamma = gamma;
    st.cur_d = (int32_t *)calloc((size_t)k, sizeof(int32_t));
    st.best = ORACLE_NEG;
    st.best_x = xs;
    st.best_d = ds;
    st.visited = 0;
    for (int x0 = 0; x0 < w; ++x0) {
        st.cur_x0 = x0;
        brute_angle_rec(&st, 0, x0);
    }
    free(st.cur_d);
    if (visited) *visited = st.visited;
    if (st.best == ORACLE_NEG) {
        for (int i = 0; i <= k; ++i) xs[i] = -1;
        for (int i = 0; i < k; ++i) ds[i] = 0;
    }
    return st.best;
}

/* The whole main problem in double: smoothing (half-width r), band FHT, the
 * angle-restricted DP and the read-back.  Returns the optimal score of the
 * smoothed image. */
double oracle_detect_angle_f64(const double *img, int h, int w, int k, int r, double gamma,
                               int32_t *xs, int32_t *ds) {
    int n = h / k;
    int W = w + n;
    double *S = (double *)malloc(sizeof(double) * (size_t)h * w);
    double *H = (double *)malloc(sizeof(double) * (size_t)k * 2 * n * W);
    double *V = (double *)malloc(sizeof(double) * (size_t)k * (2 * n - 1) * w);
    int32_t *lohi = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * n - 1));
    double s = NAN;
    if (S && H && V && lohi && oracle_gauss_rows_f64(img, h, w, r, S) == 0 &&
        oracle_angle_window(n, gamma, lohi) == 0) {
        oracle_fht_recursive_f64(S, h, w, k, H);
        oracle_dp_angle_f64(H, h, w, k, lohi, V);
        s = oracle_backtrack_angle_f64(V, h, w, k, lohi, xs, ds);
    }
    free(S);
    free(H);
    free(V);
    free(lohi);
    return s;
}

/* ---------------------------------------------------------------------------
 * Subproblems 2-3 (Sec. 2.2-2.3): the extreme polyline through a given point
 * P = (xp, j*n) on the upper border of band j (j = k: the image's bottom
 * border).  Plain definition: the maximum over all admissible polylines with
 * x_j = xp (bend limit B at every vertex, P included), the lexicographically
 * smallest among the optimal ones.  The paper builds the part below P by the
 * DP over bands j..k-1 and the part above by the same DP on the top bands
 * flipped about Ox; this oracle reaches the same optimum with one DP over
 * all bands in which every state of band j (j = k: of band k-1) whose vertex
 * on P's border is not xp is dead.  Then V_0 holds the best polylines
 * through P and the usual read-back (Eq. 5) returns the answer.
 * ------------------------------------------------------------------------ */
int oracle_dp_through_f64(const double *H, int h, int w, int k, int B, int j, int xp,
                          double *V) {
    if (k < 1 || h % k != 0 || B < 0 || j < 0 || j > k || xp < 0 || xp >= w) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    for (int b = k - 1; b >= 0; --b)
        for (int d = -(n - 1); d <= n - 1; ++d)
            for (int x = 0; x < w; ++x) {
                double *out = &V[((size_t)b * D + (d + n - 1)) * w + x];
                int xn = x + d;
                int off_point = (b == j && x != xp) || (j == k && b == k - 1 && xn != xp);
                if (xn < 0 || xn >= w || off_point) {
                    *out = ORACLE_NEG;
                    continue;
                }
                double hv = hough_at_f64(H, n, W, b, x, d);
                if (b == k - 1) {
                    *out = hv;
                    continue;
                }
                double best = ORACLE_NEG;
                for (int e = d - B; e <= d + B; ++e) {
                    if (e < -(n - 1) || e > n - 1) continue;
                    double v = V[((size_t)(b + 1) * D + (e + n - 1)) * w + xn];
                    if (v > best) best = v;
                }
                *out = (best == ORACLE_NEG) ? ORACLE_NEG : hv + best;
            }
    return 0;
}

double oracle_detect_through_f64(const double *img, int h, int w, int k, int B, int j, int xp,
                                 int32_t *xs, int32_t *ds) {
    int n = h / k;
    int W = w + n;
    double *H = (double *)malloc(sizeof(double) * (size_t)k * 2 * n * W);
    double *V = (double *)malloc(sizeof(double) * (size_t)k * (2 * n - 1) * w);
    double s = NAN;
    if (H && V) {
        oracle_fht_recursive_f64(img, h, w, k, H);
        if (oracle_dp_through_f64(H, h, w, k, B, j, xp, V) == 0)
            s = oracle_backtrack_f64(V, h, w, k, B, xs, ds);
    }
    free(H);
    free(V);
    return s;
}

/* Brute force over every admissible polyline with x_j = xp (tiny images). */
typedef struct {
    const double *img;
    int h, w, k, n, B, j, xp;
    int32_t *cur_d;
    int cur_x0;
    double best;
    int32_t *best_x;
    int32_t *best_d;
    long visited;
} brute_through_state;

static void brute_through_rec(brute_through_state *st, int i, int x) {
    if (i == st->j && x != st->xp) return;   /* vertex x_i is x */
    if (i == st->k) {
        st->visited++;
        double sc = oracle_path_score_f64(st->img, st->h, st->w, st->k, st->cur_x0, st->cur_d);
        if (sc > st->best) {
            st->best = sc;
            int xx = st->cur_x0;
            for (int q = 0; q < st->k; ++q) {
                st->best_x[q] = xx;
                st->best_d[q] = st->cur_d[q];
                xx += st->cur_d[q];
            }
            st->best_x[st->k] = xx;
        }
        return;
    }
    int n = st->n;
    for (int d = -(n - 1); d <= n - 1; ++d) {
        if (i > 0 && (d < st->cur_d[i - 1] - st->B || d > st->cur_d[i - 1] + st->B)) continue;
        if (x + d < 0 || x + d >= st->w) continue;
        st->cur_d[i] = d;
        brute_through_rec(st, i + 1, x + d);
    }
}

double oracle_brute_through_f64(const double *img, int h, int w, int k, int B, int j, int xp,
                                int32_t *xs, int32_t *ds, long *visited) {
    brute_through_state st;
    st.img = img;
    st.h = h;
    st.w = w;
    st.k = k;
    st.n = h / k;
    st.B = B;
    st.j = j;
    st.xp = xp;
    st.cur_d = (int32_t *)calloc((size_t)k, sizeof(int32_t));
    st.best = ORACLE_NEG;
    st.best_x = xs;
    st.best_d = ds;
    st.visited = 0;
    for (int x0 = 0; x0 < w; ++x0) {
        st.cur_x0 = x0;
        brute_through_rec(&st, 0, x0);
    }
    free(st.cur_d);
    if (visited) *visited = st.visited;
    if (st.best == ORACLE_NEG) {
        for (int i = 0; i <= k; ++i) xs[i] = -1;
        for (int i = 0; i < k; ++i) ds[i] = 0;
    }
    return st.best;
}

/* ---------------------------------------------------------------------------
 * Two different extreme polylines (Sec. 3, Figs. 6d and 7a; the paper does
 * not state the rule).  Reading: the first is the optimum; the second is the
 * best polyline whose top vertex x_0 lies at least `sep` columns from the
 * first's (non-maximum suppression on x_0), the lexicographically smallest
 * among its optima.  Both come from the same V: the second is the argmax of
 * V_0 over the columns |x - x_0| >= sep, read back as in Eq. 5.
 * xs: [2][k+1], ds: [2][k], scores: [2] (second: -inf and x = -1 when every
 * column is suppressed).
 * ------------------------------------------------------------------------ */
int oracle_detect_two_f64(const double *img, int h, int w, int k, int B, int sep, int32_t *xs,
                          int32_t *ds, double *scores) {
    if (k < 1 || h % k != 0 || B < 0 || sep < 1) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    double *H = (double *)malloc(sizeof(double) * (size_t)k * 2 * n * W);
    double *V = (double *)malloc(sizeof(double) * (size_t)k * D * w);
    double *V2 = (double *)malloc(sizeof(double) * (size_t)k * D * w);
    if (!H || !V || !V2) {
        free(H);
        free(V);
        free(V2);
        return -1;
    }
    oracle_fht_recursive_f64(img, h, w, k, H);
    oracle_dp_f64(H, h, w, k, B, V);
    scores[0] = oracle_backtrack_f64(V, h, w, k, B, xs, ds);
    /* the second: the same V with the suppressed top columns dead */
    memcpy(V2, V, sizeof(double) * (size_t)k * D * w);
    int x0 = xs[0];
    for (int d = 0; d < D; ++d)
        for (int x = 0; x < w; ++x)
            if (x0 >= 0 && abs(x - x0) < sep) V2[(size_t)d * w + x] = ORACLE_NEG;
    scores[1] = oracle_backtrack_f64(V2, h, w, k, B, xs + k + 1, ds + k);
    free(H);
    free(V);
    free(V2);
    return 0;
}

/* Brute force over every admissible polyline whose top vertex is at least
 * sep columns from x0 (tiny images): the best of the brute-force optima
 * through each allowed start column, taken in increasing column order. */
double oracle_brute_apart_f64(const double *img, int h, int w, int k, int B, int x0, int sep,
                              int32_t *xs, int32_t *ds) {
    double best = ORACLE_NEG;
    int32_t *bx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *bd = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    for (int i = 0; i <= k; ++i) xs[i] = -1;
    for (int i = 0; i < k; ++i) ds[i] = 0;
    for (int s0 = 0; s0 < w; ++s0) {
        if (abs(s0 - x0) < sep) continue;
        long visited = 0;
        double s = oracle_brute_through_f64(img, h, w, k, B, 0, s0, bx, bd, &visited);
        if (s > best) {
            best = s;
            for (int i = 0; i <= k; ++i) xs[i] = bx[i];
            for (int i = 0; i < k; ++i) ds[i] = bd[i];
        }
    }
    free(bx);
    free(bd);
    return best;
}

/* ---------------------------------------------------------------------------
 * Vertices in the padding (Sec. 2.2: the Hough columns run over
 * [0, w + h/k - 1]).  Each band is extended to the right by n zero columns
 * (Sec. 2.1), and the polyline's vertices may lie anywhere in [0, W),
 * W = w + n: the pixels a link covers right of the image count as zero.  The
 * DP, the read-back and the brute force below are those above with the
 * vertex domain [0, W) in place of [0, w); V: [k][2n-1][W].
 * ------------------------------------------------------------------------ */
double oracle_path_score_padded_f64(const double *img, int h, int w, int k, int x0,
                                    const int32_t *ds) {
    int n = h / k;
    int W = w + n;
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * n);
    if (!off) return ORACLE_NEG;
    oracle_off_table(n, off);
    double acc = 0.0;
    int x = x0;
    if (x < 0 || x >= W) acc = ORACLE_NEG;
    for (int i = 0; i < k && acc != ORACLE_NEG; ++i) {
        int d = ds[i];
        int s = d >= 0 ? d : -d;
        if (s > n - 1 || x + d < 0 || x + d >= W) {
            acc = ORACLE_NEG;
            break;
        }
        for (int y = 0; y < n; ++y) {
            int c = x + (d >= 0 ? 1 : -1) * off[(size_t)s * n + y];
            if (c < w) acc += img[((size_t)i * n + y) * w + c];   /* zero right of the image */
        }
        x += d;
    }
    free(off);
    return acc;
}

int oracle_dp_padded_f64(const double *H, int h, int w, int k, int B, double *V) {
    if (k < 1 || h % k != 0 || B < 0) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    for (int b = k - 1; b >= 0; --b)
        for (int d = -(n - 1); d <= n - 1; ++d)
            for (int x = 0; x < W; ++x) {
                double *out = &V[((size_t)b * D + (d + n - 1)) * W + x];
                int xn = x + d;
                if (xn < 0 || xn >= W) {
                    *out = ORACLE_NEG;
                    continue;
                }
                double hv = hough_at_f64(H, n, W, b, x, d);
                if (b == k - 1) {
                    *out = hv;
                    continue;
                }
                double best = ORACLE_NEG;
                for (int e = d - B; e <= d + B; ++e) {
                    if (e < -(n - 1) || e > n - 1) continue;
                    double v = V[((size_t)(b + 1) * D + (e + n - 1)) * W + xn];
                    if (v > best) best = v;
                }
                *out = (best == ORACLE_NEG) ? ORACLE_NEG : hv + best;
            }
    return 0;
}

double oracle_detect_padded_f64(const double *img, int h, int w, int k, int B, int32_t *xs,
                                int32_t *ds) {
    int n = h / k;
    int W = w + n;
    double *H = (double *)malloc(sizeof(double) * (size_t)k * 2 * n * W);
    double *V = (double *)malloc(sizeof(double) * (size_t)k * (2 * n - 1) * W);
    double s = NAN;
    if (H && V) {
        oracle_fht_recursive_f64(img, h, w, k, H);
        oracle_dp_padded_f64(H, h, w, k, B, V);
        /* V has W columns: the read-back over the vertex domain [0, W) is the
         * plain read-back with W as the width */
        s = oracle_backtrack_f64(V, h, W, k, B, xs, ds);
    }
    free(H);
    free(V);
    return s;
}

/* Brute force with vertices in [0, W) and zeros right of the image. */
double oracle_brute_padded_f64(const double *img, int h, int w, int k, int B, int32_t *xs,
                               int32_t *ds, long *visited) {
    int n = h / k;
    int W = w + n;
    int32_t *cd = (int32_t *)calloc((size_t)k, sizeof(int32_t));
    double best = ORACLE_NEG;
    long count = 0;
    for (int i = 0; i <= k; ++i) xs[i] = -1;
    for (int i = 0; i < k; ++i) ds[i] = 0;
    for (int x0 = 0; x0 < W; ++x0) {
        /* odometer over d in lexicographic order, pruned by the vertex domain
         * and the bend limit at the end */
        for (int i = 0; i < k; ++i) cd[i] = -(n - 1);
        for (;;) {
            int ok = 1, x = x0;
            for (int i = 0; i < k && ok; ++i) {
                if (i > 0 && (cd[i] < cd[i - 1] - B || cd[i] > cd[i - 1] + B)) ok = 0;
                x += cd[i];
                if (x < 0 || x >= W) ok = 0;
            }
            if (ok) {
                ++count;
                double sc = oracle_path_score_padded_f64(img, h, w, k, x0, cd);
                if (sc > best) {
                    best = sc;
                    int xx = x0;
                    for (int i = 0; i < k; ++i) {
                        xs[i] = xx;
                        ds[i] = cd[i];
                        xx += cd[i];
                    }
                    xs[k] = xx;
                }
            }
            int i = k - 1;
            while (i >= 0 && cd[i] == n - 1) cd[i--] = -(n - 1);
            if (i < 0) break;
            ++cd[i];
        }
    }
    free(cd);
    if (visited) *visited = count;
    return best;
}

/* ---------------------------------------------------------------------------
 * Subproblem 3 with the bend-angle window (Sec. 2.3): the extreme polyline
 * through P = (xp, j*n) whose consecutive links bend by at most gamma, on the
 * row-smoothed image (r = 0: no smoothing).  As oracle_dp_through_f64 with the
 * angle windows lohi of oracle_angle_window.
 * ------------------------------------------------------------------------ */
int oracle_dp_angle_through_f64(const double *H, int h, int w, int k, const int32_t *lohi,
                                int j, int xp, double *V) {
    if (k < 1 || h % k != 0 || j < 0 || j > k || xp < 0 || xp >= w) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    for (int b = k - 1; b >= 0; --b)
        for (int d = -(n - 1); d <= n - 1; ++d)
            for (int x = 0; x < w; ++x) {
                double *out = &V[((size_t)b * D + (d + n - 1)) * w + x];
                int xn = x + d;
                int off_point = (b == j && x != xp) || (j == k && b == k - 1 && xn != xp);
                if (xn < 0 || xn >= w || off_point) {
                    *out = ORACLE_NEG;
                    continue;
                }
                double hv = hough_at_f64(H, n, W, b, x, d);
                if (b == k - 1) {
                    *out = hv;
                    continue;
                }
                double best = ORACLE_NEG;
                for (int e = lohi[2 * (d + n - 1)]; e <= lohi[2 * (d + n - 1) + 1]; ++e) {
                    double v = V[((size_t)(b + 1) * D + (e + n - 1)) * w + xn];
                    if (v > best) best = v;
                }
                *out = (best == ORACLE_NEG) ? ORACLE_NEG : hv + best;
            }
    return 0;
}

double oracle_detect_angle_through_f64(const double *img, int h, int w, int k, int r,
                                       double gamma, int j, int xp, int32_t *xs, int32_t *ds) {
    int n = h / k;
    int W = w + n;
    double *S = (double *)malloc(sizeof(double) * (size_t)h * w);
    double *H = (double *)malloc(sizeof(double) * (size_t)k * 2 * n * W);
    double *V = (double *)malloc(sizeof(double) * (size_t)k * (2 * n - 1) * w);
    int32_t *lohi = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * n - 1));
    double s = NAN;
    if (S && H && V && lohi && oracle_gauss_rows_f64(img, h, w, r, S) == 0 &&
        oracle_angle_window(n, gamma, lohi) == 0) {
        oracle_fht_recursive_f64(S, h, w, k, H);
        if (oracle_dp_angle_through_f64(H, h, w, k, lohi, j, xp, V) == 0)
            s = oracle_backtrack_angle_f64(V, h, w, k, lohi, xs, ds);
    }
    free(S);
    free(H);
    free(V);
    free(lohi);
    return s;
}

/* Brute force: every polyline with x_j = xp whose bends pass the direct
 * angle test (tiny images; the image given is the one scored). */
typedef struct {
    const double *img;
    int h, w, k, n, j, xp;
    double gamma;
    int32_t *cur_d;
    int cur_x0;
    double best;
    int32_t *best_x;
    int32_t *best_d;
} brute_angle_through_state;

static void brute_angle_through_rec(brute_angle_through_state *st, int i, int x) {
    if (i == st->j && x != st->xp) return;
    if (i == st->k) {
        double sc = oracle_path_score_f64(st->img, st->h, st->w, st->k, st->cur_x0, st->cur_d);
        if (sc > st->best) {
            st->best = sc;
            int xx = st->cur_x0;
            for (int q = 0; q < st->k; ++q) {
                st->best_x[q] = xx;
                st->best_d[q] = st->cur_d[q];
                xx += st->cur_d[q];
            }
            st->best_x[st->k] = xx;
        }
        return;
    }
    int n = st->n;
    for (int d = -(n - 1); d <= n - 1; ++d) {
        if (i > 0 && fabs(atan((double)d / n) - atan((double)st->cur_d[i - 1] / n)) > st->gamma)
            continue;
        if (x + d < 0 || x + d >= st->w) continue;
        st->cur_d[i] = d;
        brute_angle_through_rec(st, i + 1, x + d);
    }
}

double oracle_brute_angle_through_f64(const double *img, int h, int w, int k, double gamma, int j,
                                      int xp, int32_t *xs, int32_t *ds) {
    brute_angle_through_state st;
    st.img = img;
    st.h = h;
    st.w = w;
    st.k = k;
    st.n = h / k;
    st.j = j;
    st.xp = xp;
    st.gamma = gamma;
    st.cur_d = (int32_t *)calloc((size_t)k, sizeof(int32_t));
    st.best = ORACLE_NEG;
    st.best_x = xs;
    st.best_d = ds;
    for (int i = 0; i <= k; ++i) xs[i] = -1;
    for (int i = 0; i < k; ++i) ds[i] = 0;
    for (int x0 = 0; x0 < w; ++x0) {
        st.cur_x0 = x0;
        brute_angle_through_rec(&st, 0, x0);
    }
    free(st.cur_d);
    return st.best;
}

/* ---------------------------------------------------------------------------
 * The queries of Secs. 2.2-2.3 and 3 on float32 images, in float32: the
 * decisions the library's float path takes for them.  Each is the float64
 * definition above with every value, sum and comparison in float, and the
 * Hough images from the float32 recursion (oracle_fht_recursive_f32, whose
 * summation tree the CUDA path follows).
 * ------------------------------------------------------------------------ */

/* Sec. 2.3 step 1 in float32: out(y, x) = sum over t = -r..r, in that order,
 * of (float)C(2r, r + t) * img(y, x + t), each product rounded to float and
 * added to a float accumulator that starts at 0; pixels outside the row are
 * skipped (adding their zero product would not change a float sum). */
int oracle_gauss_rows_f32(const float *img, int h, int w, int r, float *out) {
    if (r < 0) return -1;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            float acc = 0.0f;
            for (int t = -r; t <= r; ++t) {
                int c = x + t;
                if (c < 0 || c >= w) continue;
                float prod = (float)binom(2 * r, r + t) * img[(size_t)y * w + c];
                acc = acc + prod;
            }
            out[(size_t)y * w + x] = acc;
        }
    return 0;
}

/* The DP of Sec. 2.3 in float32 with per-displacement windows lohi (the
 * angle windows of oracle_angle_window) and, when j >= 0, the point P =
 * (xp, j*n) of Subproblem 3 (states off P dead, as oracle_dp_through_f64). */
static int dp_table_point_f32(const float *H, int h, int w, int k, const int32_t *lohi, int j,
                              int xp, float *V) {
    if (k < 1 || h % k != 0) return -1;
    if (j >= 0 && (j > k || xp < 0 || xp >= w)) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    for (int b = k - 1; b >= 0; --b)
        for (int d = -(n - 1); d <= n - 1; ++d)
            for (int x = 0; x < w; ++x) {
                float *out = &V[((size_t)b * D + (d + n - 1)) * w + x];
                int xn = x + d;
                int off_point =
                    j >= 0 && ((b == j && x != xp) || (j == k && b == k - 1 && xn != xp));
                if (xn < 0 || xn >= w || off_point) {
                    *out = (float)ORACLE_NEG;
                    continue;
                }
                float hv = hough_at_f32(H, n, W, b, x, d);
                if (b == k - 1) {
                    *out = hv;
                    continue;
                }
                float best = (float)ORACLE_NEG;
                for (int e = lohi[2 * (d + n - 1)]; e <= lohi[2 * (d + n - 1) + 1]; ++e) {
                    float v = V[((size_t)(b + 1) * D + (e + n - 1)) * w + xn];
                    if (v > best) best = v;
                }
                *out = (best == (float)ORACLE_NEG) ? (float)ORACLE_NEG : hv + best;
            }
    return 0;
}

int oracle_dp_angle_f32(const float *H, int h, int w, int k, const int32_t *lohi, float *V) {
    return dp_table_point_f32(H, h, w, k, lohi, -1, 0, V);
}

/* The read-back of Eq. 5 with the angle windows, in float32. */
double oracle_backtrack_angle_f32(const float *V, int h, int w, int k, const int32_t *lohi,
                                  int32_t *xs, int32_t *ds) {
    int n = h / k;
    int D = 2 * n - 1;
    float best = (float)ORACLE_NEG;
    int bx = 0, bd = 0;
    for (int x = 0; x < w; ++x)
        for (int d = -(n - 1); d <= n - 1; ++d) {
            float v = V[(size_t)(d + n - 1) * w + x];
            if (v > best) {
                best = v;
                bx = x;
                bd = d;
            }
        }
    if (best == (float)ORACLE_NEG) {
        for (int i = 0; i <= k; ++i) xs[i] = -1;
        for (int i = 0; i < k; ++i) ds[i] = 0;
        return ORACLE_NEG;
    }
    xs[0] = bx;
    ds[0] = bd;
    for (int i = 1; i < k; ++i) {
        int xi = xs[i - 1] + ds[i - 1];
        xs[i] = xi;
        int p = ds[i - 1] + n - 1;
        float bv = (float)ORACLE_NEG;
        int be = lohi[2 * p];
        for (int e = lohi[2 * p]; e <= lohi[2 * p + 1]; ++e) {
            float v = V[((size_t)i * D + (e + n - 1)) * w + xi];
            if (v > bv) {
                bv = v;
                be = e;
            }
        }
        ds[i] = be;
    }
    xs[k] = xs[k - 1] + ds[k - 1];
    return (double)best;
}

/* The main problem (j < 0) or Subproblem 3 through (xp, j*n), in float32:
 * smoothing, the float32 recursion, the windowed DP and the read-back. */
static double detect_angle_point_f32(const float *img, int h, int w, int k, int r, double gamma,
                                     int j, int xp, int32_t *xs, int32_t *ds) {
    int n = h / k;
    int W = w + n;
    float *S = (float *)malloc(sizeof(float) * (size_t)h * w);
    float *H = (float *)malloc(sizeof(float) * (size_t)k * 2 * n * W);
    float *V = (float *)malloc(sizeof(float) * (size_t)k * (2 * n - 1) * w);
    int32_t *lohi = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * n - 1));
    double s = NAN;
    if (S && H && V && lohi && oracle_gauss_rows_f32(img, h, w, r, S) == 0 &&
        oracle_angle_window(n, gamma, lohi) == 0) {
        oracle_fht_recursive_f32(S, h, w, k, H);
        if (dp_table_point_f32(H, h, w, k, lohi, j, xp, V) == 0)
            s = oracle_backtrack_angle_f32(V, h, w, k, lohi, xs, ds);
    }
    free(S);
    free(H);
    free(V);
    free(lohi);
    return s;
}

double oracle_detect_angle_f32(const float *img, int h, int w, int k, int r, double gamma,
                               int32_t *xs, int32_t *ds) {
    return detect_angle_point_f32(img, h, w, k, r, gamma, -1, 0, xs, ds);
}

double oracle_detect_angle_through_f32(const float *img, int h, int w, int k, int r,
                                       double gamma, int j, int xp, int32_t *xs, int32_t *ds) {
    if (j < 0 || j > k || xp < 0 || xp >= w) return NAN;
    return detect_angle_point_f32(img, h, w, k, r, gamma, j, xp, xs, ds);
}

/* Subproblems 2-3 with the bend limit B, in float32: the window of d is
 * [d - B, d + B] clipped to the displacement range. */
static void bend_table(int n, int B, int32_t *lohi) {
    for (int d = -(n - 1); d <= n - 1; ++d) {
        int lo = d - B, hi = d + B;
        lohi[2 * (d + n - 1)] = lo < -(n - 1) ? -(n - 1) : lo;
        lohi[2 * (d + n - 1) + 1] = hi > n - 1 ? n - 1 : hi;
    }
}

double oracle_detect_through_f32(const float *img, int h, int w, int k, int B, int j, int xp,
                                 int32_t *xs, int32_t *ds) {
    if (k < 1 || h % k != 0 || B < 0 || j < 0 || j > k || xp < 0 || xp >= w) return NAN;
    int n = h / k;
    int W = w + n;
    float *H = (float *)malloc(sizeof(float) * (size_t)k * 2 * n * W);
    float *V = (float *)malloc(sizeof(float) * (size_t)k * (2 * n - 1) * w);
    int32_t *lohi = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * n - 1));
    double s = NAN;
    if (H && V && lohi) {
        bend_table(n, B, lohi);
        oracle_fht_recursive_f32(img, h, w, k, H);
        if (dp_table_point_f32(H, h, w, k, lohi, j, xp, V) == 0)
            s = oracle_backtrack_f32(V, h, w, k, B, xs, ds);
    }
    free(H);
    free(V);
    free(lohi);
    return s;
}

/* Vertices in the padding (Sec. 2.2), float32: the DP over the vertex
 * domain [0, W) as oracle_dp_padded_f64, and the read-back with W as the
 * width. */
int oracle_dp_padded_f32(const float *H, int h, int w, int k, int B, float *V) {
    if (k < 1 || h % k != 0 || B < 0) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    for (int b = k - 1; b >= 0; --b)
        for (int d = -(n - 1); d <= n - 1; ++d)
            for (int x = 0; x < W; ++x) {
                float *out = &V[((size_t)b * D + (d + n - 1)) * W + x];
                int xn = x + d;
                if (xn < 0 || xn >= W) {
                    *out = (float)ORACLE_NEG;
                    continue;
                }
                float hv = hough_at_f32(H, n, W, b, x, d);
                if (b == k - 1) {
                    *out = hv;
                    continue;
                }
                float best = (float)ORACLE_NEG;
                for (int e = d - B; e <= d + B; ++e) {
                    if (e < -(n - 1) || e > n - 1) continue;
                    float v = V[((size_t)(b + 1) * D + (e + n - 1)) * W + xn];
                    if (v > best) best = v;
                }
                *out = (best == (float)ORACLE_NEG) ? (float)ORACLE_NEG : hv + best;
            }
    return 0;
}

double oracle_detect_padded_f32(const float *img, int h, int w, int k, int B, int32_t *xs,
                                int32_t *ds) {
    int n = h / k;
    int W = w + n;
    float *H = (float *)malloc(sizeof(float) * (size_t)k * 2 * n * W);
    float *V = (float *)malloc(sizeof(float) * (size_t)k * (2 * n - 1) * W);
    double s = NAN;
    if (H && V) {
        oracle_fht_recursive_f32(img, h, w, k, H);
        oracle_dp_padded_f32(H, h, w, k, B, V);
        s = oracle_backtrack_f32(V, h, W, k, B, xs, ds);
    }
    free(H);
    free(V);
    return s;
}

/* Two different extreme polylines (Sec. 3), float32: as
 * oracle_detect_two_f64 on the float32 V. */
int oracle_detect_two_f32(const float *img, int h, int w, int k, int B, int sep, int32_t *xs,
                          int32_t *ds, double *scores) {
    if (k < 1 || h % k != 0 || B < 0 || sep < 1) return -1;
    int n = h / k;
    int W = w + n;
    int D = 2 * n - 1;
    float *H = (float *)malloc(sizeof(float) * (size_t)k * 2 * n * W);
    float *V = (float *)malloc(sizeof(float) * (size_t)k * D * w);
    float *V2 = (float *)malloc(sizeof(float) * (size_t)k * D * w);
    if (!H || !V || !V2) {
        free(H);
        free(V);
        free(V2);
        return -1;
    }
    oracle_fht_recursive_f32(img, h, w, k, H);
    oracle_dp_f32(H, h, w, k, B, V);
    scores[0] = oracle_backtrack_f32(V, h, w, k, B, xs, ds);
    memcpy(V2, V, sizeof(float) * (size_t)k * D * w);
    int x0 = xs[0];
    for (int d = 0; d < D; ++d)
        for (int x = 0; x < w; ++x)
            if (x0 >= 0 && abs(x - x0) < sep) V2[(size_t)d * w + x] = (float)ORACLE_NEG;
    scores[1] = oracle_backtrack_f32(V2, h, w, k, B, xs + k + 1, ds + k);
    free(H);
    free(V);
    free(V2);
    return 0;
}
