/*
 * lse_oracle.c -- plain FP64 CPU oracle for the two fast level set evolutions
 * (LSE) of Li, Shi, Wang and Miao, "Extracting Man-Made Objects From Remote
 * Sensing Images via Fast Level Set Evolutions" (arXiv 1409.7474).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously correct statement of
 * what the GPU library computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA path (it does not even include the library's
 * public header) and the CUDA path never calls it.
 *
 * Everything is double precision, row-major, pixel (y, x) at y*W + x; a
 * multi-band image is band-planar: band b, pixel (y, x) at (b*H + y)*W + x.
 * Where the build enables OpenMP, the two per-pixel maps (the update and the
 * convolution) and the maximum max|D| spread their pixels over threads; every
 * pixel is still computed by one thread in the order written here, and a
 * maximum does not depend on the order it is taken in, so results do not
 * depend on the thread count.  Every sum over pixels (region statistics,
 * counts) stays one sequential loop.
 *
 * What each piece follows in the paper:
 *   gaussian taps ........ G_sigma of Table I step 4 / Sec. III-D Step 4: the
 *                          sampled, normalised TS x TS Gaussian (no truncation
 *                          of tiny tails).
 *   gradient ............. |grad phi| of Eqs. 14 and 17, discretised as the
 *                          edge-based MATLAB listing does: unit-spacing central
 *                          differences inside, one-sided differences on the
 *                          first/last row and column, zero along a dimension of
 *                          size 1.
 *   conv_same ............ "G_sigma * phi" (Table I step 4) as the listing's
 *                          'same'-size convolution with zero padding.
 *   edge indicator ....... g(I) = 1 / (1 + |grad(G_sigma1 * I)|^2), Eq. 14
 *                          (definition carried over from Eq. 2).  Multi-band
 *                          input is first reduced to the equal-weight band mean
 *                          and scaled by edge_scale (the listing works on
 *                          0..255 intensities).
 *   region statistics .... c+ and c- of Eq. 15: means of I over phi >= 0 and
 *                          phi < 0 (per band for vector images).
 *   region force ......... R_Td of Eq. 17: D / max|D| with
 *                          D = sum_b (c+_b - c-_b)(2 I_b - c+_b - c-_b).
 *                          Eq. 16 prints (c+ + c-) in the first factor; expanding
 *                          Eq. 15 with lambda = 1 gives (c+ - c-), which Eq. 17
 *                          and Table I also print, so the minus is used.
 *                          The sum over bands is the vector-valued Chan-Vese
 *                          form the paper cites for its notation ([78]), with
 *                          every lambda equal to 1.
 *   update ............... Eq. 18: u = phi + dt * R * |grad phi|.
 *   regularisation ....... Table I step 4: v = G_sigma * u.
 *   re-initialisation .... Table I step 3 / Step 3: phi = +1 where v >= 0,
 *                          -1 elsewhere (the listing's tie rule: v = 0 -> +1),
 *                          applied after smoothing as the listing orders it.
 *   stopping ............. Step 5: a fixed iteration count, with an optional
 *                          early stop once fewer than early_stop_frac * H * W
 *                          pixels change sign in one iteration.
 *
 * Two variants, reached through the *_variant / *_padded entry points (the
 * plain entry points are the method as read above):
 *   Table I order ........ Table I lists update (step 2), re-initialisation
 *                          (step 3), then regularisation (step 4): on a
 *                          re-initialising iteration u is binarised first
 *                          (u >= 0 -> +1, the same tie rule) and v = G * that;
 *                          the next iteration starts from v itself.
 *   replicate padding .... the convolution takes the nearest image value
 *                          outside the image instead of 0.
 *
 * Degenerate cases the paper leaves open: when phi >= 0 holds nowhere or
 * everywhere, when the two sides' means agree to within rounding, or when
 * max|D| = 0, the region force is taken as R = 0 (the iteration only smooths)
 * and the degenerate flag is raised.  "Agree to within rounding" means
 * max_b |c+_b - c-_b| <= 1e-6 * max_b (|c+_b| + |c-_b|): without this rule a
 * constant image, whose exact D is zero, would have its rounding noise
 * normalised by Eq. 17 into a full-strength random force.  The mean of an
 * empty side is reported as 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the per-pixel maps (OpenMP builds): 0 = the OpenMP default. */
static int g_threads = 0;

void oracle_set_threads(int n) { g_threads = n > 0 ? n : 0; }

static int oracle_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORACLE_TERM_REGION 0
#define ORACLE_TERM_EDGE 1
#define ORACLE_ORDER_LISTING 0  /* update, smooth, re-initialise */
#define ORACLE_ORDER_TABLE1 1   /* update, re-initialise, smooth */
#define ORACLE_PAD_ZERO 0
#define ORACLE_PAD_REPLICATE 1
#define ORACLE_MAX_BANDS 8
/* Relative contrast below which c+ and c- count as equal (see above). */
#define ORACLE_CONTRAST_TOL 1e-6

typedef struct {
    int iterations_run;
    long long last_flips;      /* sign changes in the last iteration run */
    long long area_plus;       /* |{v_final >= 0}| */
    double c_plus[ORACLE_MAX_BANDS];  /* Eq. 15 means over the final mask */
    double c_minus[ORACLE_MAX_BANDS];
    double norm;               /* max|D| used by the last iteration (region) */
    int degenerate;            /* some iteration had R = 0 by the rule above */
} oracle_stats;

/* ------------------------------------------------------------------ */
/* Gaussian kernel G_sigma (Table I step 4).                          */
/* ------------------------------------------------------------------ */
void oracle_gaussian_taps(double sigma, int ts, double *G)
{
    int r = (ts - 1) / 2;
    double total = 0.0;
    for (int i = -r; i <= r; ++i)
        for (int j = -r; j <= r; ++j) {
            double w = exp(-(double)(i * i + j * j) / (2.0 * sigma * sigma));
            G[(i + r) * ts + (j + r)] = w;
            total += w;
        }
    for (int k = 0; k < ts * ts; ++k)
        G[k] /= total;
}

/* ------------------------------------------------------------------ */
/* Gradient as the listing's `gradient`: x runs along a row.          */
/* ------------------------------------------------------------------ */
static double grad_x_at(const double *f, int H, int W, int y, int x)
{
    const double *row = f + (size_t)y * W;
    (void)H;
    if (W == 1) return 0.0;
    if (x == 0) return row[1] - row[0];
    if (x == W - 1) return row[W - 1] - row[W - 2];
    return 0.5 * (row[x + 1] - row[x - 1]);
}

static double grad_y_at(const double *f, int H, int W, int y, int x)
{
    if (H == 1) return 0.0;
    if (y == 0) return f[(size_t)W + x] - f[x];
    if (y == H - 1) return f[(size_t)(H - 1) * W + x] - f[(size_t)(H - 2) * W + x];
    return 0.5 * (f[(size_t)(y + 1) * W + x] - f[(size_t)(y - 1) * W + x]);
}

void oracle_gradient(const double *f, int H, int W, double *fx, double *fy)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            fx[(size_t)y * W + x] = grad_x_at(f, H, W, y, x);
            fy[(size_t)y * W + x] = grad_y_at(f, H, W, y, x);
        }
}

/* ------------------------------------------------------------------ */
/* 'same'-size 2-D convolution.                                       */
/* out(y,x) = sum_{i,j} G(i,j) f(y - i, x - j), i,j in [-r, r], with  */
/* f = 0 outside the image (pad = ORACLE_PAD_ZERO) or f = its nearest */
/* image value there (ORACLE_PAD_REPLICATE).                          */
/* ------------------------------------------------------------------ */
static double conv_at(const double *f, int H, int W, const double *G, int ts,
                      int y, int x, int pad)
{
    int r = (ts - 1) / 2;
    double acc = 0.0;
    for (int i = -r; i <= r; ++i) {
        int yy = y - i;
        if (yy < 0 || yy >= H) {
            if (pad == ORACLE_PAD_ZERO) continue;
            yy = yy < 0 ? 0 : H - 1;
        }
        for (int j = -r; j <= r; ++j) {
            int xx = x - j;
            if (xx < 0 || xx >= W) {
                if (pad == ORACLE_PAD_ZERO) continue;
                xx = xx < 0 ? 0 : W - 1;
            }
            acc += G[(i + r) * ts + (j + r)] * f[(size_t)yy * W + xx];
        }
    }
    return acc;
}

void oracle_conv_same_padded(const double *f, int H, int W, const double *G, int ts,
                             int pad, double *out)
{
    /* each output pixel is one thread's own sum, taken in the order above */
#pragma omp parallel for schedule(static) num_threads(oracle_threads()) \
    if ((size_t)H * W >= 65536)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            out[(size_t)y * W + x] = conv_at(f, H, W, G, ts, y, x, pad);
}

void oracle_conv_same(const double *f, int H, int W, const double *G, int ts,
                      double *out)
{
    oracle_conv_same_padded(f, H, W, G, ts, ORACLE_PAD_ZERO, out);
}

/* ------------------------------------------------------------------ */
/* Edge indicator g(I) of Eq. 14, computed once per image.           */
/* ------------------------------------------------------------------ */
void oracle_edge_indicator(const double *I, int H, int W, int B, double sigma1,
                           int ts1, double edge_scale, double *g)
{
    size_t N = (size_t)H * W;
    double *J = (double *)malloc(N * sizeof(double));
    double *S = (double *)malloc(N * sizeof(double));
    double *G1 = (double *)malloc((size_t)ts1 * ts1 * sizeof(double));
    for (size_t p = 0; p < N; ++p) {
        double acc = 0.0;
        for (int b = 0; b < B; ++b)
            acc += I[(size_t)b * N + p];
        J[p] = edge_scale * (acc / B);
    }
    oracle_gaussian_taps(sigma1, ts1, G1);
    oracle_conv_same(J, H, W, G1, ts1, S);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double sx = grad_x_at(S, H, W, y, x);
            double sy = grad_y_at(S, H, W, y, x);
            g[(size_t)y * W + x] = 1.0 / (1.0 + sx * sx + sy * sy);
        }
    free(J);
    free(S);
    free(G1);
}

/* ------------------------------------------------------------------ */
/* Region statistics c+ / c- (Eq. 15).  Returns |{phi >= 0}|.         */
/* ------------------------------------------------------------------ */
long long oracle_region_stats(const double *I, int H, int W, int B,
                              const double *phi, double *c_plus,
                              double *c_minus)
{
    size_t N = (size_t)H * W;
    long long n_plus = 0;
    for (size_t p = 0; p < N; ++p)
        if (phi[p] >= 0.0) ++n_plus;
    long long n_minus = (long long)N - n_plus;
    for (int b = 0; b < B; ++b) {
        double s_plus = 0.0, s_minus = 0.0;
        const double *Ib = I + (size_t)b * N;
        for (size_t p = 0; p < N; ++p) {
            if (phi[p] >= 0.0) s_plus += Ib[p];
            else s_minus += Ib[p];
        }
        c_plus[b] = n_plus > 0 ? s_plus / (double)n_plus : 0.0;
        c_minus[b] = n_minus > 0 ? s_minus / (double)n_minus : 0.0;
    }
    return n_plus;
}

/* ------------------------------------------------------------------ */
/* One evaluation context: the current LSF and the quantities that    */
/* the per-pixel update of Eq. 18 needs.                              */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *I;
    const double *g;
    const double *phi;
    int H, W, B, term;
    double dt;
    double c_plus[ORACLE_MAX_BANDS], c_minus[ORACLE_MAX_BANDS];
    double norm;        /* max|D| (region) */
    int zero_force;     /* R = 0 everywhere (degenerate region case) */
} step_ctx;

/* D(y,x) = sum_b (c+_b - c-_b)(2 I_b - c+_b - c-_b): numerator of Eq. 17. */
static double region_numerator_at(const step_ctx *c, size_t p)
{
    size_t N = (size_t)c->H * c->W;
    double d = 0.0;
    for (int b = 0; b < c->B; ++b) {
        double cp = c->c_plus[b], cm = c->c_minus[b];
        d += (cp - cm) * (2.0 * c->I[(size_t)b * N + p] - cp - cm);
    }
    return d;
}

/* Fills the global quantities: c+/c- and max|D| for the region term.     */
static void prepare_ctx(step_ctx *c)
{
    size_t N = (size_t)c->H * c->W;
    c->norm = 0.0;
    c->zero_force = 0;
    if (c->term != ORACLE_TERM_REGION) return;
    long long n_plus = oracle_region_stats(c->I, c->H, c->W, c->B, c->phi,
                                           c->c_plus, c->c_minus);
    if (n_plus == 0 || n_plus == (long long)N) {
        c->zero_force = 1;
        return;
    }
    double contrast = 0.0, scale = 0.0;
    for (int b = 0; b < c->B; ++b) {
        double d = fabs(c->c_plus[b] - c->c_minus[b]);
        double a = fabs(c->c_plus[b]) + fabs(c->c_minus[b]);
        if (d > contrast) contrast = d;
        if (a > scale) scale = a;
    }
    if (contrast <= ORACLE_CONTRAST_TOL * scale) {
        c->zero_force = 1;
        return;
    }
    double m = 0.0;
    /* a maximum does not depend on the order it is taken in */
#pragma omp parallel for reduction(max : m) schedule(static) \
    num_threads(oracle_threads()) if (N >= 65536)
    for (size_t p = 0; p < N; ++p) {
        double a = fabs(region_numerator_at(c, p));
        if (a > m) m = a;
    }
    c->norm = m;
    if (m == 0.0) c->zero_force = 1;
}

/* Data term R at pixel p: R_Td (Eq. 17) or E_Td = g (Eq. 14). */
static double force_at(const step_ctx *c, size_t p)
{
    if (c->term == ORACLE_TERM_EDGE) return c->g[p];
    if (c->zero_force) return 0.0;
    return region_numerator_at(c, p) / c->norm;
}

/* Explicit update of Eq. 18 at (y, x): u = phi + dt * R * |grad phi|. */
static double update_at(const step_ctx *c, int y, int x)
{
    double fx = grad_x_at(c->phi, c->H, c->W, y, x);
    double fy = grad_y_at(c->phi, c->H, c->W, y, x);
    size_t p = (size_t)y * c->W + x;
    return c->phi[p] + c->dt * force_at(c, p) * sqrt(fx * fx + fy * fy);
}

static void fill_ctx(step_ctx *c, const double *I, int H, int W, int B,
                     int term, const double *g, const double *phi, double dt)
{
    c->I = I;
    c->g = g;
    c->phi = phi;
    c->H = H;
    c->W = W;
    c->B = B;
    c->term = term;
    c->dt = dt;
    prepare_ctx(c);
}

/* u over the whole image (no smoothing): exposed for the tests. */
int oracle_update(const double *I, int H, int W, int B, int term,
                  const double *g, const double *phi, double dt, double *u)
{
    step_ctx c;
    fill_ctx(&c, I, H, W, B, term, g, phi, dt);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            u[(size_t)y * W + x] = update_at(&c, y, x);
    return c.zero_force;
}

/* R over the whole image, with c+/c- and max|D|: exposed for the tests. */
int oracle_region_force(const double *I, int H, int W, int B,
                        const double *phi, double *R, double *norm,
                        double *c_plus, double *c_minus)
{
    step_ctx c;
    fill_ctx(&c, I, H, W, B, ORACLE_TERM_REGION, NULL, phi, 0.0);
    size_t N = (size_t)H * W;
    if (R)
        for (size_t p = 0; p < N; ++p)
            R[p] = force_at(&c, p);
    *norm = c.norm;
    for (int b = 0; b < B; ++b) {
        c_plus[b] = c.c_plus[b];
        c_minus[b] = c.c_minus[b];
    }
    return c.zero_force;
}

/* One iteration: u = phi + dt R |grad phi| (Eq. 18); in the Table I order
 * on a re-initialising iteration u -> (u >= 0 ? 1 : -1) (Table I step 3);
 * v = G_sigma * u with the given padding (Table I step 4).  The listing's
 * re-initialisation of v is the caller's.  Returns 1 when the region force
 * was zero by the degenerate rule. */
int oracle_step_variant(const double *I, int H, int W, int B, int term,
                        const double *g, const double *phi, double dt, double sigma,
                        int ts, int order, int reinit, int pad, double *v,
                        double *norm_out, double *c_plus, double *c_minus)
{
    size_t N = (size_t)H * W;
    double *u = (double *)malloc(N * sizeof(double));
    double *G = (double *)malloc((size_t)ts * ts * sizeof(double));
    step_ctx c;
    fill_ctx(&c, I, H, W, B, term, g, phi, dt);
#pragma omp parallel for schedule(static) num_threads(oracle_threads()) \
    if (N >= 65536)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            u[(size_t)y * W + x] = update_at(&c, y, x);
    if (order == ORACLE_ORDER_TABLE1 && reinit)
        for (size_t p = 0; p < N; ++p) u[p] = u[p] >= 0.0 ? 1.0 : -1.0;
    oracle_gaussian_taps(sigma, ts, G);
    oracle_conv_same_padded(u, H, W, G, ts, pad, v);
    if (norm_out) *norm_out = c.norm;
    if (c_plus && c_minus)
        for (int b = 0; b < B; ++b) {
            c_plus[b] = c.c_plus[b];
            c_minus[b] = c.c_minus[b];
        }
    free(u);
    free(G);
    return c.zero_force;
}

/* One iteration without re-initialisation: v = G_sigma * (phi + dt R |grad phi|),
 * zero padding. */
int oracle_step(const double *I, int H, int W, int B, int term,
                const double *g, const double *phi, double dt, double sigma,
                int ts, double *v, double *norm_out, double *c_plus,
                double *c_minus)
{
    return oracle_step_variant(I, H, W, B, term, g, phi, dt, sigma, ts,
                               ORACLE_ORDER_LISTING, 0, ORACLE_PAD_ZERO, v, norm_out,
                               c_plus, c_minus);
}

/* One iteration (listing order, zero padding, not re-initialised) with the
 * region statistics given instead of taken from phi: c+ / c- per band and
 * the normaliser M (Eq. 17), as a row strip of a larger image steps with the
 * whole image's statistics.  zero_force: R = 0.  The edge term ignores them. */
void oracle_step_given(const double *I, int H, int W, int B, int term, const double *g,
                       const double *phi, double dt, double sigma, int ts,
                       const double *c_plus, const double *c_minus, double norm,
                       int zero_force, double *v)
{
    size_t N = (size_t)H * W;
    double *u = (double *)malloc(N * sizeof(double));
    double *G = (double *)malloc((size_t)ts * ts * sizeof(double));
    step_ctx c;
    c.I = I;
    c.g = g;
    c.phi = phi;
    c.H = H;
    c.W = W;
    c.B = B;
    c.term = term;
    c.dt = dt;
    for (int b = 0; b < B; ++b) {
        c.c_plus[b] = c_plus[b];
        c.c_minus[b] = c_minus[b];
    }
    c.norm = norm;
    c.zero_force = zero_force || !(norm > 0.0);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            u[(size_t)y * W + x] = update_at(&c, y, x);
    oracle_gaussian_taps(sigma, ts, G);
    oracle_conv_same(u, H, W, G, ts, v);
    free(u);
    free(G);
}

/* The same iteration evaluated only at n sample pixels (ys[k], xs[k]).
 * The global quantities (c+/c-, max|D|) are still computed over the whole
 * image; u is evaluated on the window each sample needs.  For checks of
 * large images where a full FP64 step would take too long. */
int oracle_step_sampled(const double *I, int H, int W, int B, int term,
                        const double *g, const double *phi, double dt,
                        double sigma, int ts, int n, const int *ys,
                        const int *xs, double *v_samples, double *norm_out,
                        double *c_plus, double *c_minus)
{
    int r = (ts - 1) / 2;
    double *G = (double *)malloc((size_t)ts * ts * sizeof(double));
    step_ctx c;
    fill_ctx(&c, I, H, W, B, term, g, phi, dt);
    oracle_gaussian_taps(sigma, ts, G);
    for (int k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int i = -r; i <= r; ++i) {
            int yy = ys[k] - i;
            if (yy < 0 || yy >= H) continue;
            for (int j = -r; j <= r; ++j) {
                int xx = xs[k] - j;
                if (xx < 0 || xx >= W) continue;
                acc += G[(i + r) * ts + (j + r)] * update_at(&c, yy, xx);
            }
        }
        v_samples[k] = acc;
    }
    if (norm_out) *norm_out = c.norm;
    if (c_plus && c_minus)
        for (int b = 0; b < B; ++b) {
            c_plus[b] = c.c_plus[b];
            c_minus[b] = c.c_minus[b];
        }
    free(G);
    return c.zero_force;
}

/* Is iteration n (0-based) followed by re-initialisation to the binary LSF?
 * period 1: every iteration (the listing); 0: never; k: after iterations
 * k-1, 2k-1, ... (Step 3 says "periodically"). */
static int reinit_after(int n, int period)
{
    if (period == 1) return 1;
    if (period <= 0) return 0;
    return ((n + 1) % period) == 0;
}

/* The whole evolution (Table I steps 2-6) in the given step order and
 * padding.  Returns 0, or -1 on bad input.  v_out receives the last smoothed
 * LSF v (in the listing's order: before its re-initialisation);
 * mask_out[p] = (v_out[p] >= 0). */
int oracle_evolve_variant(const double *I, int H, int W, int B, int term,
                          const double *g, const double *phi0, double dt,
                          double sigma, int ts, int iterations, int reinit_period,
                          double early_stop_frac, int order, int pad, double *v_out,
                          unsigned char *mask_out, oracle_stats *st)
{
    if (H < 1 || W < 1 || B < 1 || B > ORACLE_MAX_BANDS || ts < 1 ||
        (ts % 2) == 0 || iterations < 1)
        return -1;
    if (term == ORACLE_TERM_EDGE && g == NULL) return -1;
    size_t N = (size_t)H * W;
    double *phi = (double *)malloc(N * sizeof(double));
    memcpy(phi, phi0, N * sizeof(double));
    memset(st, 0, sizeof(*st));
    for (int n = 0; n < iterations; ++n) {
        double norm = 0.0;
        const int reinit_n = reinit_after(n, reinit_period);
        st->degenerate |= oracle_step_variant(I, H, W, B, term, g, phi, dt, sigma, ts,
                                              order, reinit_n, pad, v_out, &norm, NULL,
                                              NULL) &&
                          term == ORACLE_TERM_REGION;
        st->norm = norm;
        long long flips = 0;
        for (size_t p = 0; p < N; ++p)
            if ((v_out[p] >= 0.0) != (phi[p] >= 0.0)) ++flips;
        st->last_flips = flips;
        st->iterations_run = n + 1;
        /* in the Table I order the re-initialisation came before smoothing */
        int reinit = reinit_n && order == ORACLE_ORDER_LISTING;
        for (size_t p = 0; p < N; ++p)
            phi[p] = reinit ? (v_out[p] >= 0.0 ? 1.0 : -1.0) : v_out[p];
        if (early_stop_frac > 0.0 && (double)flips < early_stop_frac * (double)N)
            break;
    }
    for (size_t p = 0; p < N; ++p)
        mask_out[p] = v_out[p] >= 0.0 ? 1 : 0;
    if (term == ORACLE_TERM_REGION)
        st->area_plus = oracle_region_stats(I, H, W, B, v_out, st->c_plus,
                                            st->c_minus);
    else {
        long long a = 0;
        for (size_t p = 0; p < N; ++p) a += mask_out[p];
        st->area_plus = a;
    }
    free(phi);
    return 0;
}

/* The evolution in the listing's order with zero padding. */
int oracle_evolve(const double *I, int H, int W, int B, int term,
                  const double *g, const double *phi0, double dt,
                  double sigma, int ts, int iterations, int reinit_period,
                  double early_stop_frac, double *v_out,
                  unsigned char *mask_out, oracle_stats *st)
{
    return oracle_evolve_variant(I, H, W, B, term, g, phi0, dt, sigma, ts, iterations,
                                 reinit_period, early_stop_frac, ORACLE_ORDER_LISTING,
                                 ORACLE_PAD_ZERO, v_out, mask_out, st);
}
