/*
 * FP64 CPU oracle for the Quantile Rendering (Q-Render) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load or call this library; the CUDA
 * library never does, and the two share no code, headers or tables.  Both
 * sides receive the same seeded inputs from the input generator.
 *
 * What it computes, in double precision, following the paper:
 *   - Sec. 3: a 3D Gaussian has covariance Sigma = R S S^T R^T from its scale
 *     s (S = diag(exp(log_scale))) and rotation quaternion; it is splatted to
 *     the image with EWA splatting (the local affine approximation J of the
 *     perspective projection at the mean, Sigma' = J W Sigma W^T J^T);
 *     alpha'_i = alpha_i * G_i(u) with G the projected Gaussian at pixel u.
 *   - Eq. 1 (volume rendering, "V-Render"): w_i = T_i alpha'_i,
 *     T_i = prod_{j<i} (1 - alpha'_j), summed over the depth-ordered list S_r.
 *   - Sec. 4.2 / Algorithm 1 (QuantileRender): transmittance partitioned into
 *     K+1 equal segments; a Gaussian whose test transmittance crosses the next
 *     boundary 1-(k+1)/(K+1) is a quantile Gaussian and is alpha-blended with
 *     the quantile transmittance T^Q; the walk stops once the test
 *     transmittance is below 1/(K+1); the result is divided by 1 - T^Q.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the index list I of a pixel is every Gaussian in front of the near
 *     plane with alpha' >= alpha_min (1/255), sorted by camera-space depth,
 *     ties by lower index; no tiles are involved here;
 *   - alpha' = min(alpha_max, alpha * G) with alpha_max = 0.99;
 *   - the EWA covariance gets "dilation" px^2 added to its diagonal;
 *   - the dense blend stops before a Gaussian that would take T below T_min
 *     (T_min = 0 gives Eq. 1 over the whole list);
 *   - a pixel with no quantile Gaussian (1 - T^Q = 0) renders zero.
 *
 * Brute force on purpose: every pixel evaluates every Gaussian.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOMEM 2

/* ------------------------------------------------------------------------ */
/* Sec. 3: rotation from a quaternion (w, x, y, z), normalised first.         */
/* ------------------------------------------------------------------------ */
void or_quat_to_rotation(const float q_in[4], double R[9])
{
    double w = q_in[0], x = q_in[1], y = q_in[2], z = q_in[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Sigma = R S S^T R^T with S = diag(exp(log_scale)); out row-major 3x3. */
void or_covariance3d(const float log_scale[3], const float quat[4], double Sigma[9])
{
    double R[9], M[9];
    or_quat_to_rotation(quat, R);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            M[r * 3 + c] = R[r * 3 + c] * exp((double)log_scale[c]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += M[r * 3 + k] * M[c * 3 + k];
            Sigma[r * 3 + c] = s;
        }
}

/*
 * Projection of every Gaussian (Sec. 3, EWA splatting).
 * cam = [R(9) row-major world->camera, t(3), fx, fy, cx, cy, near] (float32).
 * Outputs (double): mean2d [n][2], conic [n][3] = (A00, A01, A11) of
 * A = Sigma'^{-1}, cov2d [n][3] = (S00, S01, S11) of Sigma' (with dilation),
 * depth [n] = camera-space z of the mean; valid [n] = 1 if z > near and
 * det Sigma' > 0.
 */
int or_project(int64_t n, const float *mean, const float *log_scale, const float *quat,
               const float *cam, double dilation,
               double *mean2d, double *conic, double *cov2d, double *depth, int32_t *valid)
{
    if (n < 0 || !mean || !log_scale || !quat || !cam) return OR_ERR_ARG;
    double W[9], tw[3];
    for (int i = 0; i < 9; ++i) W[i] = cam[i];
    for (int i = 0; i < 3; ++i) tw[i] = cam[9 + i];
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15], znear = cam[16];
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {mean[3 * i], mean[3 * i + 1], mean[3 * i + 2]};
        double c[3];
        for (int r = 0; r < 3; ++r)
            c[r] = W[r * 3] * p[0] + W[r * 3 + 1] * p[1] + W[r * 3 + 2] * p[2] + tw[r];
        depth[i] = c[2];
        mean2d[2 * i] = mean2d[2 * i + 1] = 0.0;
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0.0;
        cov2d[3 * i] = cov2d[3 * i + 1] = cov2d[3 * i + 2] = 0.0;
        valid[i] = 0;
        if (!(c[2] > znear)) continue;
        double Sigma[9];
        or_covariance3d(log_scale + 3 * i, quat + 4 * i, Sigma);
        /* J: Jacobian of (fx x/z + cx, fy y/z + cy) at the camera-space mean */
        double z = c[2];
        double J[6] = {fx / z, 0.0, -fx * c[0] / (z * z),
                       0.0, fy / z, -fy * c[1] / (z * z)};
        double T[6]; /* T = J W */
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k)
                T[r * 3 + k] = J[r * 3] * W[k] + J[r * 3 + 1] * W[3 + k] + J[r * 3 + 2] * W[6 + k];
        double V[4]; /* Sigma' = T Sigma T^T */
        for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s) {
                double acc = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        acc += T[r * 3 + a] * Sigma[a * 3 + b] * T[s * 3 + b];
                V[r * 2 + s] = acc;
            }
        double s00 = V[0] + dilation, s01 = 0.5 * (V[1] + V[2]), s11 = V[3] + dilation;
        double det = s00 * s11 - s01 * s01;
        if (!(det > 0.0)) continue;
        cov2d[3 * i] = s00; cov2d[3 * i + 1] = s01; cov2d[3 * i + 2] = s11;
        conic[3 * i] = s11 / det; conic[3 * i + 1] = -s01 / det; conic[3 * i + 2] = s00 / det;
        mean2d[2 * i] = fx * c[0] / z + cx;
        mean2d[2 * i + 1] = fy * c[1] / z + cy;
        valid[i] = 1;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on one depth-ordered list of alpha' values.                    */
/* ------------------------------------------------------------------------ */
/*
 * a[0..n)  : alpha' of the list I, front to back.
 * sel[i]   : 1 if Gaussian i is a quantile Gaussian.
 * w[i]     : its blend weight T^Q * alpha'_i before normalisation (0 if not).
 * *TQ      : final quantile transmittance T^Q.
 * *n_proc  : how many list entries the walk visited before stopping.
 * Returns the number of quantile Gaussians.
 */
int or_qrender_list(int64_t n, const double *a, int K, int32_t *sel, double *w,
                    double *TQ, int64_t *n_proc)
{
    double T = 1.0, Tq = 1.0;
    int k = 0, m = 0;
    int64_t i;
    for (i = 0; i < n; ++i) { sel[i] = 0; w[i] = 0.0; }
    for (i = 0; i < n; ++i) {
        double Ttest = T * (1.0 - a[i]);
        if (Ttest < 1.0 - (double)(k + 1) / (double)(K + 1)) {
            k = k + 1;
            w[i] = Tq * a[i];
            sel[i] = 1;
            ++m;
            Tq = Tq * (1.0 - a[i]);
            while (Ttest < 1.0 - (double)(k + 1) / (double)(K + 1)) k = k + 1;
        }
        if (Ttest < 1.0 / (double)(K + 1)) { ++i; break; }
        T = Ttest;
    }
    if (TQ) *TQ = Tq;
    if (n_proc) *n_proc = i;
    return m;
}

/* n(t) = #{ j in 1..K : t < 1 - j/(K+1) }: how many segment boundaries lie above t. */
static int crossed(double t, int K)
{
    int c = 0;
    for (int j = 1; j <= K; ++j)
        if (t < 1.0 - (double)j / (double)(K + 1)) ++c;
    return c;
}

/*
 * The same selection written as a closed form over the full transmittance
 * sequence T_0 = 1, T_i = T_{i-1}(1 - a_i): Gaussian i is visited iff every
 * earlier T stayed >= 1/(K+1), and it is a quantile Gaussian iff it is
 * visited and n(T_i) > n(T_{i-1}).
 */
int or_qselect_closed_form(int64_t n, const double *a, int K, int32_t *sel)
{
    double Tprev = 1.0;
    int visited = 1, m = 0;
    for (int64_t i = 0; i < n; ++i) {
        double Ti = Tprev * (1.0 - a[i]);
        sel[i] = (visited && crossed(Ti, K) > crossed(Tprev, K)) ? 1 : 0;
        m += sel[i];
        if (visited && Ti < 1.0 / (double)(K + 1)) visited = 0;
        Tprev = Ti;
    }
    return m;
}

/*
 * App. C reads Algorithm 1 as a right Riemann sum over the transmittance
 * domain split into K + 1 equal segments: each boundary 1 - k/(K+1) that the
 * accumulated transmittance crosses contributes the feature of the Gaussian
 * at which it is crossed, with the segment width 1/(K+1).  Reading (the
 * optional weight form of the select rules): the same walk and selection as
 * or_qrender_list; a quantile Gaussian's weight is the number of boundaries
 * its test transmittance crosses, and the render divides by the number
 * crossed in all, so the weights sum to 1 like Algorithm 1's normalised ones.
 * sel[i] = 1 for the quantile Gaussians, w[i] their crossing counts; *n_proc
 * as or_qrender_list.  Returns the number of quantile Gaussians.
 */
int or_riemann_list(int64_t n, const double *a, int K, int32_t *sel, double *w, int64_t *n_proc)
{
    double T = 1.0;
    int k = 0, m = 0;
    int64_t i;
    for (i = 0; i < n; ++i) { sel[i] = 0; w[i] = 0.0; }
    for (i = 0; i < n; ++i) {
        double Ttest = T * (1.0 - a[i]);
        if (Ttest < 1.0 - (double)(k + 1) / (double)(K + 1)) {
            int k0 = k;
            k = k + 1;
            while (Ttest < 1.0 - (double)(k + 1) / (double)(K + 1)) k = k + 1;
            if (k > K) k = K;              /* the K boundaries 1 - j/(K+1), j = 1..K */
            w[i] = (double)(k - k0);
            sel[i] = 1;
            ++m;
        }
        if (Ttest < 1.0 / (double)(K + 1)) { ++i; break; }
        T = Ttest;
    }
    if (n_proc) *n_proc = i;
    return m;
}

/*
 * Eq. 1 on one list: w_i = T_i alpha'_i with T_i the transmittance before i.
 * With T_min > 0 the walk stops before the Gaussian whose test transmittance
 * would fall below T_min.  Returns the number of blended Gaussians.
 */
int64_t or_dense_list(int64_t n, const double *a, double T_min, double *w, double *T_final)
{
    double T = 1.0;
    int64_t i, used = 0;
    for (i = 0; i < n; ++i) w[i] = 0.0;
    for (i = 0; i < n; ++i) {
        double Ttest = T * (1.0 - a[i]);
        if (T_min > 0.0 && Ttest < T_min) break;
        w[i] = T * a[i];
        ++used;
        T = Ttest;
    }
    if (T_final) *T_final = T;
    return used;
}

/* ------------------------------------------------------------------------ */
/* Top-K: the comparison renderer of Sec. 4.2 and Table 1 (complexity table). */
/* ------------------------------------------------------------------------ */
/*
 * The paper's top-K renderer sorts the Gaussians of a ray by weight and keeps
 * the K largest.  Reading: the weights are Eq. 1's w_i = T_i alpha'_i over the
 * list I (the dense walk, with its T_min stop), equal weights keep the
 * earlier entry, and the kept Gaussians are blended with their Eq. 1 weights
 * normalised by their sum (as Algorithm 1 normalises by 1 - T^Q).
 * Streaming selection along the walk: at most K kept entries; once K are
 * kept, a strictly larger weight replaces the smallest kept one (the latest
 * of equal ones).  sel[i] = 1 for the kept entries and w[i] their Eq. 1
 * weights (0 elsewhere); *n_used receives the entries the walk blended.
 * Returns the number kept, or -1 when out of memory.
 */
int or_topk_list(int64_t n, const double *a, int K, double T_min, int32_t *sel, double *w,
                 int64_t *n_used)
{
    int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
    if (!kept) return -1;
    double T = 1.0;
    int m = 0;
    int64_t i;
    for (i = 0; i < n; ++i) { sel[i] = 0; w[i] = 0.0; }
    for (i = 0; i < n; ++i) {
        double Ttest = T * (1.0 - a[i]);
        if (T_min > 0.0 && Ttest < T_min) break;
        w[i] = T * a[i];
        if (m < K) {
            kept[m++] = i;
        } else {
            int s = 0;
            for (int j = 1; j < K; ++j)
                if (w[kept[j]] < w[kept[s]] || (w[kept[j]] == w[kept[s]] && kept[j] > kept[s])) s = j;
            if (w[i] > w[kept[s]]) kept[s] = i;
        }
        T = Ttest;
    }
    if (n_used) *n_used = i;
    for (int j = 0; j < m; ++j) sel[kept[j]] = 1;
    for (int64_t l = 0; l < n; ++l)
        if (!sel[l]) w[l] = 0.0;
    free(kept);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Stratified-K: the two-pass adaptive variant of App. E.                     */
/* ------------------------------------------------------------------------ */
/* Standard normal CDF, Phi(z) = erfc(-z / sqrt 2) / 2. */
static double normal_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* Phi^{-1}(p) for p in (0, 1) by bisection on Phi (slow, to full precision). */
static double normal_inv(double p)
{
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 400 && hi - lo > 1e-15 * (1.0 + fabs(lo)); ++it) {
        double mid = 0.5 * (lo + hi);
        if (normal_cdf(mid) < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/*
 * App. E, "Stratified-sampling": pass 1 walks the list as Eq. 1 does (T_min
 * stop) and takes the mean mu and the standard deviation sigma of the
 * transmittances T_1..T_n after each blended Gaussian.  Reading of the
 * appendix: the K boundaries are spaced uniformly in the probability of
 * N(mu, sigma^2) over the transmittance interval [0, 1] and mapped back,
 *     u_lo = Phi(-mu / sigma),  u_hi = Phi((1 - mu) / sigma),
 *     tau_k = mu + sigma Phi^{-1}(u_lo + (u_hi - u_lo)(1 - k/(K+1))),  k = 1..K,
 * so they crowd where the transmittances do; with fewer than two blended
 * Gaussians (sigma = 0) they are Algorithm 1's 1 - k/(K+1).  Pass 2 is
 * Algorithm 1 with tau_k in place of 1 - k/(K+1): a Gaussian whose test
 * transmittance falls below the next boundary is kept with weight T^Q alpha',
 * and the walk stops once the test transmittance falls below tau_K.
 * Outputs as or_qrender_list; tau (nullable) receives tau_1..tau_K and
 * stats (nullable) (mu, sigma, n).  Returns the number kept, -1 without memory.
 */
int or_stratified_list(int64_t n, const double *a, int K, double T_min, int32_t *sel, double *w,
                       double *TQ, int64_t *n_proc, double *tau, double *stats)
{
    double *Tv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *th = (double *)malloc(sizeof(double) * (size_t)(K + 1));
    if (!Tv || !th) { free(Tv); free(th); return -1; }
    /* pass 1: the transmittances of the dense walk */
    double T = 1.0;
    int64_t nb = 0;
    for (int64_t i = 0; i < n; ++i) {
        double Ttest = T * (1.0 - a[i]);
        if (T_min > 0.0 && Ttest < T_min) break;
        T = Ttest;
        Tv[nb++] = T;
    }
    double mu = 0.0, var = 0.0;
    for (int64_t i = 0; i < nb; ++i) mu += Tv[i];
    mu = nb > 0 ? mu / (double)nb : 0.0;
    for (int64_t i = 0; i < nb; ++i) var += (Tv[i] - mu) * (Tv[i] - mu);
    var = nb > 0 ? var / (double)nb : 0.0;
    double sigma = sqrt(var);
    for (int k = 1; k <= K; ++k) {
        double c = 1.0 - (double)k / (double)(K + 1);
        if (nb >= 2 && sigma > 0.0) {
            double ulo = normal_cdf(-mu / sigma), uhi = normal_cdf((1.0 - mu) / sigma);
            th[k] = mu + sigma * normal_inv(ulo + (uhi - ulo) * c);
        } else {
            th[k] = c;
        }
        if (tau) tau[k - 1] = th[k];
    }
    if (stats) { stats[0] = mu; stats[1] = sigma; stats[2] = (double)nb; }
    /* pass 2: Algorithm 1 with the boundaries tau_k */
    double Tq = 1.0;
    int k = 0, m = 0;
    int64_t i;
    T = 1.0;
    for (i = 0; i < n; ++i) { sel[i] = 0; w[i] = 0.0; }
    for (i = 0; i < n; ++i) {
        double Ttest = T * (1.0 - a[i]);
        if (k < K && Ttest < th[k + 1]) {
            k = k + 1;
            w[i] = Tq * a[i];
            sel[i] = 1;
            ++m;
            Tq = Tq * (1.0 - a[i]);
            while (k < K && Ttest < th[k + 1]) k = k + 1;
        }
        if (Ttest < th[K]) { ++i; break; }
        T = Ttest;
    }
    if (TQ) *TQ = Tq;
    if (n_proc) *n_proc = i;
    free(Tv); free(th);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel renderer (brute force over all Gaussians).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double depth;
    int64_t id;
    double a;        /* alpha' (clamped) */
    double g;        /* alpha * G, unclamped */
    double G;        /* Gaussian value exp(-q/2) */
    double dx, dy;   /* pixel centre minus projected mean */
    double qabs;     /* conditioning magnitude of q (for the tie check) */
} member_t;

static int member_cmp(const void *pa, const void *pb)
{
    const member_t *a = (const member_t *)pa, *b = (const member_t *)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->id < b->id) ? -1 : (a->id > b->id);
}

typedef struct {
    /* inputs */
    int64_t n;
    const double *mean2d, *conic, *depth, *alpha;
    const int32_t *valid;
    const double *feat; int C;
    int K; double alpha_min, alpha_max, T_min;
    double tie_eps;                 /* relative alpha' error the tie check allows */
    int64_t npix; const int32_t *pix;
    const double *grad_out;         /* backward only */
    /* outputs */
    double *out_q; int32_t *ids; double *wq; int32_t *cnt; double *tq;
    double *out_dense; double *t_final; int32_t *n_members; int32_t *n_proc; int32_t *tie;
    int32_t *members; int max_members;   /* optional: I(p) in depth order, -1 padded */
    double *scale_q, *scale_dense;       /* optional: sum_j |w_j| max|f_j| (error denominators) */
    int32_t *n_dense;                    /* optional: entries the dense walk blended */
    int rule;                            /* or_render_rule: RULE_TOPK, RULE_STRATIFIED, RULE_RIEMANN */
    double *tau_out;                     /* or_render_rule: [npix][K] boundaries (stratified) */
    /* threading */
    int tid, nthreads; int status;
} render_job_t;

typedef struct {
    member_t *m; int64_t cap, len;
    double *border; int64_t bcap, blen;    /* depths of Gaussians with alpha*G near alpha_min */
    double *a, *w, *wd; int32_t *sel; int64_t acap;
} scratch_t;

static int grow(void **p, int64_t *cap, int64_t need, size_t elem)
{
    if (need <= *cap) return 0;
    int64_t nc = *cap ? *cap : 256;
    while (nc < need) nc *= 2;
    void *q = realloc(*p, (size_t)nc * elem);
    if (!q) return -1;
    *p = q; *cap = nc;
    return 0;
}

/*
 * Relative FP32 error bound of alpha * G at one (pixel, Gaussian) pair that the
 * near-tie classifier allows: tie_eps (1 + qabs) + 4u, with qabs the
 * conditioning magnitude of q (see classify_ties).
 */
static double alpha_rel_err(double tie_eps, double qabs)
{
    return tie_eps * (1.0 + qabs) + 4.0 * ldexp(1.0, -24);
}

/* Add one candidate (a Gaussian evaluated at the pixel) to the pixel's list
 * state: it is a member of I(p) when alpha' = min(alpha_max, g) >= alpha_min;
 * its depth is also recorded as a border depth when g lies within the FP32
 * error of alpha_min (for the tie check).  Returns 0 on success. */
static int add_candidate(const render_job_t *J, scratch_t *S, double depth, int64_t id, double g,
                         double G, double dx, double dy, double qabs)
{
    double rel = alpha_rel_err(J->tie_eps, qabs);
    /* alpha*G within the FP32 error of alpha_min: |ln(g / alpha_min)| <= 4 rel */
    if (J->tie && g > 0.0 && fabs(log(g / J->alpha_min)) <= 4.0 * rel) {
        if (grow((void **)&S->border, &S->bcap, S->blen + 1, sizeof(double))) return -1;
        S->border[S->blen++] = depth;
    }
    double a = g < J->alpha_max ? g : J->alpha_max;   /* alpha' = min(alpha_max, alpha G) */
    if (a < J->alpha_min) return 0;
    if (grow((void **)&S->m, &S->cap, S->len + 1, sizeof(member_t))) return -1;
    member_t *mm = &S->m[S->len++];
    mm->depth = depth; mm->id = id; mm->g = g; mm->G = G;
    mm->a = a;
    mm->dx = dx; mm->dy = dy; mm->qabs = qabs;
    return 0;
}

/* Order the members by (depth, id) (Sec. 3, the ordered sequence) and lay out
 * their alpha' values front to back.  Returns 0 on success. */
static int finish_list(scratch_t *S)
{
    qsort(S->m, (size_t)S->len, sizeof(member_t), member_cmp);
    if (grow((void **)&S->a, &S->acap, S->len + 1, sizeof(double))) return -1;
    S->w = (double *)realloc(S->w, (size_t)S->acap * sizeof(double));
    S->wd = (double *)realloc(S->wd, (size_t)S->acap * sizeof(double));
    S->sel = (int32_t *)realloc(S->sel, (size_t)S->acap * sizeof(int32_t));
    if (!S->w || !S->wd || !S->sel) return -1;
    for (int64_t j = 0; j < S->len; ++j) S->a[j] = S->m[j].a;
    return 0;
}

/* Build the depth-ordered list I(p) of one pixel.  Returns 0 on success. */
static int build_list(const render_job_t *J, scratch_t *S, int px, int py)
{
    double ux = px + 0.5, uy = py + 0.5;
    S->len = 0; S->blen = 0;
    for (int64_t i = 0; i < J->n; ++i) {
        /* a Gaussian with a non-finite parameter contributes nothing (the
         * projection marks non-finite geometry invalid; the opacity here) */
        if (!J->valid[i] || !isfinite(J->alpha[i])) continue;
        double dx = ux - J->mean2d[2 * i], dy = uy - J->mean2d[2 * i + 1];
        double A00 = J->conic[3 * i], A01 = J->conic[3 * i + 1], A11 = J->conic[3 * i + 2];
        double q = A00 * dx * dx + 2.0 * A01 * dx * dy + A11 * dy * dy;
        double G = exp(-0.5 * q);
        double g = J->alpha[i] * G;
        /* conditioning of q for an FP32 sum-of-squares evaluation along the
         * conic's principal axes: |d| sqrt(lambda_max(A)) sqrt(q) + q */
        double lmax = 0.5 * (A00 + A11) + sqrt(0.25 * (A00 - A11) * (A00 - A11) + A01 * A01);
        double qabs = sqrt(dx * dx + dy * dy) * sqrt(lmax > 0.0 ? lmax : 0.0) * sqrt(q > 0.0 ? q : 0.0) + fabs(q);
        if (add_candidate(J, S, J->depth[i], i, g, G, dx, dy, qabs)) return -1;
    }
    return finish_list(S);
}

/*
 * Near-tie classification of one pixel (parity diagnostics, not rendering).
 * A GPU that evaluates alpha' in FP32 may take a different branch than this
 * FP64 walk only where a decision is closer to its threshold than the FP32
 * error can reach.  The GPU evaluates q/2 = (d.w1)^2 + (d.w2)^2 with the
 * conic's principal axes w rounded to FP32; the relative error of its alpha'_i
 * is bounded by tie_eps * (1 + |d| sqrt(lambda_max(A) q) + q) + 4u
 * (u = 2^-24), and that of a transmittance product accumulates a_i/(1-a_i)
 * times it plus two roundings per factor.
 * Bits for Algorithm 1: 1 = a visited test transmittance within that error of
 * a segment boundary; 2 = a Gaussian up to the stopping point with alpha*G
 * within error of alpha_min; 4 = two visited list entries whose depths are
 * within FP32 resolution.  For the dense blend, up to its stopping point:
 * 8 = a test transmittance within error of T_min, 64 = the alpha_min border,
 * 128 = equal depths (16 is unused).  An alpha' clamped at alpha_max counts
 * as exact only where alpha*G exceeds alpha_max by more than its error.
 */
static int classify_ties(const render_job_t *J, const scratch_t *S, int64_t nproc_q,
                         int64_t nused_dense)
{
    const double u = ldexp(1.0, -24);
    int flags = 0, K = J->K;
    double T = 1.0, E = 0.0;
    int64_t last_q = nproc_q - 1;                       /* index of the last visited entry */
    int64_t last_d = nused_dense < S->len ? nused_dense : S->len - 1;
    for (int64_t i = 0; i < S->len; ++i) {
        const member_t *m = &S->m[i];
        double rel = alpha_rel_err(J->tie_eps, m->qabs);
        /* the clamp alpha' = alpha_max is exact only when alpha*G clears it by
         * more than its error; within that error the FP32 clamp may fall
         * either way and 1 - alpha' carries the error of an unclamped value */
        double ea = (m->g * (1.0 - rel) >= J->alpha_max) ? 0.0 : rel * m->a / (1.0 - m->a);
        E += ea + 2.0 * u;
        double Tt = T * (1.0 - m->a);
        if (i <= last_q)
            for (int j = 0; j < K; ++j) {
                double tau = 1.0 - (double)(j + 1) / (double)(K + 1);
                if (fabs(Tt - tau) <= (2.0 * E + 2.0 * u) * tau) flags |= 1;
            }
        if (i + 1 < S->len) {
            double z0 = m->depth, z1 = S->m[i + 1].depth;
            int close = fabs(z1 - z0) <= 4.0 * u * fabs(z0);
            if (close && i <= last_q) flags |= 4;
            if (close && i <= last_d) flags |= 128;
        }
        if (i <= last_d && J->T_min > 0.0 &&
            fabs(Tt - J->T_min) <= (2.0 * E + 2.0 * u) * J->T_min) flags |= 8;
        T = Tt;
    }
    /* a Gaussian at the alpha_min border matters if it lies before the stop */
    double zq = (last_q >= 0 && last_q < S->len - 1) ? S->m[last_q].depth : INFINITY;
    double zd = (last_d >= 0 && last_d < S->len - 1) ? S->m[last_d].depth : INFINITY;
    for (int64_t b = 0; b < S->blen; ++b) {
        if (S->border[b] <= zq * (1.0 + 4.0 * u)) flags |= 2;
        if (S->border[b] <= zd * (1.0 + 4.0 * u)) flags |= 64;
    }
    return flags;
}

/*
 * The near-tie classification of one pixel from its candidates, for tests
 * that pin the classifier on hand-built lists.  Candidate c is a Gaussian
 * evaluated at the pixel: camera depth[c], index id[c], g[c] = alpha * G
 * (unclamped) and the conditioning magnitude qabs[c] of its q.  The list I is
 * built exactly as for a rendered pixel (membership, border depths, order),
 * Algorithm 1 and the dense walk run on it, and the classifier's flags are
 * returned; n_proc / n_used (nullable) receive the entries Algorithm 1
 * visited and the entries the dense walk blended.  Returns -1 on bad
 * arguments or memory exhaustion.
 */
int or_classify_candidates(int64_t n, const double *depth, const int64_t *id, const double *g,
                           const double *qabs, int K, double alpha_min, double alpha_max,
                           double T_min, double tie_eps, int64_t *n_proc, int64_t *n_used)
{
    if (n < 0 || K < 1 || !depth || !id || !g || !qabs) return -1;
    render_job_t J;
    memset(&J, 0, sizeof(J));
    int32_t tie_dummy = 0;
    J.K = K; J.alpha_min = alpha_min; J.alpha_max = alpha_max; J.T_min = T_min;
    J.tie_eps = tie_eps; J.tie = &tie_dummy;
    scratch_t S;
    memset(&S, 0, sizeof(S));
    int flags = -1;
    for (int64_t c = 0; c < n; ++c)
        if (add_candidate(&J, &S, depth[c], id[c], g[c], 1.0, 0.0, 0.0, qabs[c])) goto done;
    if (finish_list(&S)) goto done;
    {
        double Tq = 1.0, Tf = 1.0;
        int64_t nproc = 0;
        or_qrender_list(S.len, S.a, K, S.sel, S.w, &Tq, &nproc);
        int64_t nused = or_dense_list(S.len, S.a, T_min, S.wd, &Tf);
        if (n_proc) *n_proc = nproc;
        if (n_used) *n_used = nused;
        flags = classify_ties(&J, &S, nproc, nused);
    }
done:
    free(S.m); free(S.border); free(S.a); free(S.w); free(S.wd); free(S.sel);
    return flags;
}

#define RULE_TOPK 1
#define RULE_STRATIFIED 2
#define RULE_RIEMANN 3

/*
 * Near-tie classification for the two select rules of or_render_rule, with
 * the error model of classify_ties.  Bits: 2 = an alpha_min border entry, 4 =
 * equal depths, 8 = the T_min decision, all up to the last entry either walk
 * visits; 1 = the rule's own decision:
 *   top-K: the K-th and (K+1)-th largest weights w = T alpha' within their
 *     FP32 errors (relative E_T + rel(alpha') + u each);
 *   stratified: a visited test transmittance of pass 2 within its error plus
 *     the error of the boundary tau_k.  The boundary is computed in FP32 from
 *     mu and sigma of pass 1's transmittances (whose errors E_n T_n give
 *     d mu <= mean E_n T_n, d var <= 2 mean |T_n - mu| E_n T_n), with the
 *     normal CDF and its inverse within a few units in the last place:
 *     d tau_k <= d mu + |z_k| d sigma + sigma d z_k + 2u |tau_k|,
 *     d z_k = 16u |z_k| + 64u / phi(z_k).
 */
static int classify_rule_ties(const render_job_t *J, const scratch_t *S, int rule, int64_t nproc,
                              int64_t nused, const double *tau, const double *stats)
{
    const double u = ldexp(1.0, -24);
    int flags = 0, K = J->K;
    int64_t last_d = nused < S->len ? nused : S->len - 1;
    int64_t last_q = nproc - 1;
    int64_t last = last_d > last_q ? last_d : last_q;
    double T = 1.0, E = 0.0;
    double *wv = NULL, *we = NULL;
    if (rule == RULE_TOPK) {
        wv = (double *)malloc(sizeof(double) * (size_t)(S->len + 1));
        we = (double *)malloc(sizeof(double) * (size_t)(S->len + 1));
        if (!wv || !we) { free(wv); free(we); return 255; }
    }
    /* pass-1 statistics errors (stratified) */
    double dmu = 0.0, dvar = 0.0;
    double mu = stats ? stats[0] : 0.0, sigma = stats ? stats[1] : 0.0;
    int64_t nb = stats ? (int64_t)stats[2] : 0;
    for (int64_t i = 0; i < S->len; ++i) {
        const member_t *m = &S->m[i];
        double rel = alpha_rel_err(J->tie_eps, m->qabs);
        int exact = m->g * (1.0 - rel) >= J->alpha_max;
        double ea = exact ? 0.0 : rel * m->a / (1.0 - m->a);
        double Tt = T * (1.0 - m->a);
        if (rule == RULE_TOPK && i < nused) {
            wv[i] = T * m->a;
            we[i] = E + (exact ? 0.0 : rel) + u;      /* relative error of fl32(T a) */
        }
        E += ea + 2.0 * u;
        /* the T_min decision, up to and including the entry that stopped the walk */
        if (i <= last_d && J->T_min > 0.0 && fabs(Tt - J->T_min) <= (2.0 * E + 2.0 * u) * J->T_min)
            flags |= 8;
        if (i < nused && i < nb) {
            dmu += E * Tt;
            dvar += 2.0 * fabs(Tt - mu) * E * Tt;
        }
        T = Tt;
    }
    if (rule == RULE_STRATIFIED && nb >= 2 && sigma > 0.0) {
        dmu /= (double)nb;
        double dsigma = dvar / (double)nb / (2.0 * sigma) + 2.0 * u * sigma;
        T = 1.0; E = 0.0;
        for (int64_t i = 0; i <= last_q && i < S->len; ++i) {
            const member_t *m = &S->m[i];
            double rel = alpha_rel_err(J->tie_eps, m->qabs);
            double ea = (m->g * (1.0 - rel) >= J->alpha_max) ? 0.0 : rel * m->a / (1.0 - m->a);
            E += ea + 2.0 * u;
            double Tt = T * (1.0 - m->a);
            for (int k = 0; k < K; ++k) {
                double z = (tau[k] - mu) / sigma;
                double phi = exp(-0.5 * z * z) / sqrt(2.0 * 3.14159265358979323846);
                double dz = 16.0 * u * fabs(z) + 64.0 * u / phi;
                double dtau = dmu + fabs(z) * dsigma + sigma * dz + 2.0 * u * fabs(tau[k]);
                if (fabs(Tt - tau[k]) <= (2.0 * E + 2.0 * u) * tau[k] + 2.0 * dtau) flags |= 1;
            }
            T = Tt;
        }
    } else if (rule == RULE_STRATIFIED || rule == RULE_RIEMANN) {
        /* uniform boundaries (Algorithm 1's): the checks of classify_ties */
        T = 1.0; E = 0.0;
        for (int64_t i = 0; i <= last_q && i < S->len; ++i) {
            const member_t *m = &S->m[i];
            double rel = alpha_rel_err(J->tie_eps, m->qabs);
            double ea = (m->g * (1.0 - rel) >= J->alpha_max) ? 0.0 : rel * m->a / (1.0 - m->a);
            E += ea + 2.0 * u;
            double Tt = T * (1.0 - m->a);
            for (int k = 0; k < K; ++k)
                if (fabs(Tt - tau[k]) <= (2.0 * E + 2.0 * u) * tau[k]) flags |= 1;
            T = Tt;
        }
    }
    if (rule == RULE_TOPK && nused > K) {
        /* the K-th and (K+1)-th largest weights: sort (weight desc, position asc) */
        int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)nused);
        if (!ord) { free(wv); free(we); return 255; }
        for (int64_t i = 0; i < nused; ++i) ord[i] = i;
        for (int64_t i = 1; i < nused; ++i) {          /* insertion sort: small lists */
            int64_t v = ord[i], j = i;
            while (j > 0 && (wv[ord[j - 1]] < wv[v] || (wv[ord[j - 1]] == wv[v] && ord[j - 1] > v))) {
                ord[j] = ord[j - 1];
                --j;
            }
            ord[j] = v;
        }
        int64_t p = ord[K - 1], q = ord[K];
        if (fabs(wv[p] - wv[q]) <= 2.0 * (we[p] * wv[p] + we[q] * wv[q])) flags |= 1;
        free(ord);
    }
    free(wv); free(we);
    for (int64_t i = 0; i + 1 < S->len && i <= last; ++i)
        if (fabs(S->m[i + 1].depth - S->m[i].depth) <= 4.0 * u * fabs(S->m[i].depth)) flags |= 4;
    double zl = (last >= 0 && last < S->len - 1) ? S->m[last].depth : INFINITY;
    for (int64_t b = 0; b < S->blen; ++b)
        if (S->border[b] <= zl * (1.0 + 4.0 * u)) flags |= 2;
    return flags;
}

/* One pixel under a select rule of or_render_rule. */
static int render_rule_pixel(render_job_t *J, scratch_t *S, int64_t p)
{
    const int K = J->K, C = J->C;
    double Tq = 1.0, stats[3] = {0.0, 0.0, 0.0};
    int64_t nproc = 0, nused = 0;
    double *tau = (double *)malloc(sizeof(double) * (size_t)K);
    if (!tau) return -1;
    int m;
    double D;
    if (J->rule == RULE_TOPK) {
        m = or_topk_list(S->len, S->a, K, J->T_min, S->sel, S->w, &nused);
        nproc = nused;
        D = 0.0;                             /* normalisation: divide by the kept sum */
        for (int64_t i = 0; i < S->len; ++i) D += S->w[i];
        Tq = 1.0 - D;
    } else if (J->rule == RULE_RIEMANN) {
        m = or_riemann_list(S->len, S->a, K, S->sel, S->w, &nproc);
        nused = nproc;
        D = 0.0;                             /* the boundaries crossed in all */
        for (int64_t i = 0; i < S->len; ++i) D += S->w[i];
        Tq = 1.0 - D / (double)(K + 1);
        for (int k = 1; k <= K; ++k) tau[k - 1] = 1.0 - (double)k / (double)(K + 1);
    } else {
        m = or_stratified_list(S->len, S->a, K, J->T_min, S->sel, S->w, &Tq, &nproc, tau, stats);
        double Tf = 1.0;
        nused = or_dense_list(S->len, S->a, J->T_min, S->wd, &Tf);
        if (J->tau_out)
            for (int k = 0; k < K; ++k) J->tau_out[p * K + k] = tau[k];
    }
    if (m < 0) { free(tau); return -1; }
    if (J->rule == RULE_STRATIFIED) D = 1.0 - Tq;
    if (J->cnt) J->cnt[p] = m;
    if (J->n_proc) J->n_proc[p] = (int32_t)nproc;
    if (J->tq) J->tq[p] = Tq;
    int j = 0;
    for (int64_t i = 0; i < S->len && j < K; ++i)
        if (S->sel[i]) {
            if (J->ids) J->ids[p * K + j] = (int32_t)S->m[i].id;
            if (J->wq) J->wq[p * K + j] = S->w[i] / D;
            ++j;
        }
    for (; j < K; ++j) {
        if (J->ids) J->ids[p * K + j] = -1;
        if (J->wq) J->wq[p * K + j] = 0.0;
    }
    if (J->out_q && J->feat) {
        double *o = J->out_q + p * C;
        double sc = 0.0;
        for (int c = 0; c < C; ++c) o[c] = 0.0;
        if (m > 0)
            for (int64_t i = 0; i < S->len; ++i)
                if (S->sel[i]) {
                    const double *f = J->feat + S->m[i].id * C;
                    double mx = 0.0;
                    for (int c = 0; c < C; ++c) {
                        o[c] += S->w[i] / D * f[c];
                        mx = fabs(f[c]) > mx ? fabs(f[c]) : mx;
                    }
                    sc += fabs(S->w[i] / D) * mx;
                }
        if (J->scale_q) J->scale_q[p] = sc;
    }
    if (J->tie)
        J->tie[p] = classify_rule_ties(J, S, J->rule, nproc, nused, tau,
                                       J->rule == RULE_STRATIFIED ? stats : NULL);
    free(tau);
    return 0;
}

static void *render_rule_worker(void *arg)
{
    render_job_t *J = (render_job_t *)arg;
    scratch_t S;
    memset(&S, 0, sizeof(S));
    for (int64_t p = J->tid; p < J->npix; p += J->nthreads) {
        int px = J->pix[2 * p], py = J->pix[2 * p + 1];
        if (build_list(J, &S, px, py) || render_rule_pixel(J, &S, p)) {
            J->status = OR_ERR_NOMEM;
            break;
        }
        if (J->n_members) J->n_members[p] = (int32_t)S.len;
    }
    free(S.m); free(S.border); free(S.a); free(S.w); free(S.wd); free(S.sel);
    return NULL;
}

static void *render_worker(void *arg)
{
    render_job_t *J = (render_job_t *)arg;
    scratch_t S;
    memset(&S, 0, sizeof(S));
    const int K = J->K, C = J->C;
    for (int64_t p = J->tid; p < J->npix; p += J->nthreads) {
        int px = J->pix[2 * p], py = J->pix[2 * p + 1];
        if (build_list(J, &S, px, py)) { J->status = OR_ERR_NOMEM; break; }
        if (J->n_members) J->n_members[p] = (int32_t)S.len;
        if (J->members)
            for (int j = 0; j < J->max_members; ++j)
                J->members[p * J->max_members + j] = j < S.len ? (int32_t)S.m[j].id : -1;
        /* Algorithm 1 */
        double Tq = 1.0; int64_t nproc = 0;
        int m = or_qrender_list(S.len, S.a, K, S.sel, S.w, &Tq, &nproc);
        if (J->n_proc) J->n_proc[p] = (int32_t)nproc;
        if (J->tq) J->tq[p] = Tq;
        if (J->cnt) J->cnt[p] = m;
        double D = 1.0 - Tq;
        if (J->ids || J->wq) {
            int j = 0;
            for (int64_t i = 0; i < S.len && j < K; ++i)
                if (S.sel[i]) {
                    if (J->ids) J->ids[p * K + j] = (int32_t)S.m[i].id;
                    if (J->wq) J->wq[p * K + j] = S.w[i] / D;
                    ++j;
                }
            for (; j < K; ++j) {
                if (J->ids) J->ids[p * K + j] = -1;
                if (J->wq) J->wq[p * K + j] = 0.0;
            }
        }
        if (J->out_q && J->feat) {
            double *o = J->out_q + p * C;
            for (int c = 0; c < C; ++c) o[c] = 0.0;
            if (m > 0) {
                for (int64_t i = 0; i < S.len; ++i)
                    if (S.sel[i]) {
                        const double *f = J->feat + S.m[i].id * C;
                        for (int c = 0; c < C; ++c) o[c] += S.w[i] * f[c];
                    }
                for (int c = 0; c < C; ++c) o[c] = o[c] / D;
            }
        }
        if (J->scale_q && J->feat) {
            double sc = 0.0;
            for (int64_t i = 0; i < S.len; ++i)
                if (S.sel[i]) {
                    const double *f = J->feat + S.m[i].id * C;
                    double mx = 0.0;
                    for (int c = 0; c < C; ++c) mx = fabs(f[c]) > mx ? fabs(f[c]) : mx;
                    sc += fabs(S.w[i] / D) * mx;
                }
            J->scale_q[p] = sc;
        }
        /* Eq. 1 */
        int64_t nused = S.len;
        if (J->out_dense || J->t_final || J->tie || J->n_dense) {
            double Tf = 1.0;
            nused = or_dense_list(S.len, S.a, J->T_min, S.wd, &Tf);
            if (J->t_final) J->t_final[p] = Tf;
            if (J->out_dense && J->feat) {
                double *o = J->out_dense + p * C;
                double sc = 0.0;
                for (int c = 0; c < C; ++c) o[c] = 0.0;
                for (int64_t i = 0; i < S.len; ++i)
                    if (S.wd[i] != 0.0) {
                        const double *f = J->feat + S.m[i].id * C;
                        double mx = 0.0;
                        for (int c = 0; c < C; ++c) {
                            o[c] += S.wd[i] * f[c];
                            mx = fabs(f[c]) > mx ? fabs(f[c]) : mx;
                        }
                        sc += S.wd[i] * mx;
                    }
                if (J->scale_dense) J->scale_dense[p] = sc;
            }
        }
        if (J->n_dense) J->n_dense[p] = (int32_t)nused;
        if (J->tie) J->tie[p] = classify_ties(J, &S, nproc, nused);
    }
    free(S.m); free(S.border); free(S.a); free(S.w); free(S.wd); free(S.sel);
    return NULL;
}

/*
 * Render the pixels listed in pix [npix][2] = (x, y).  Every output pointer
 * may be NULL.  feat is [n][C] in double (already decoded).  Outputs:
 * out_q [npix][C] (Algorithm 1, normalised), ids/wq [npix][K] (quantile
 * Gaussians in depth order and their normalised weights, -1 / 0 padded),
 * cnt, tq = T^Q, out_dense [npix][C] (Eq. 1), t_final, n_members = |I(p)|,
 * n_proc = entries visited by Algorithm 1, tie = near-tie flags, members
 * [npix][max_members] = the first max_members entries of I(p) (-1 padded),
 * scale_q / scale_dense [npix] = sum over blended Gaussians of
 * |weight| * max_c |f_c| (the denominators of the parity error metric),
 * n_dense [npix] = entries the dense walk blended.
 */
int or_render(int64_t n, const double *mean2d, const double *conic, const double *depth,
              const double *alpha, const int32_t *valid, const double *feat, int C,
              int K, double alpha_min, double alpha_max, double T_min, double tie_eps,
              int64_t npix, const int32_t *pix, int nthreads,
              double *out_q, int32_t *ids, double *wq, int32_t *cnt, double *tq,
              double *out_dense, double *t_final, int32_t *n_members, int32_t *n_proc,
              int32_t *tie, int32_t *members, int max_members, double *scale_q,
              double *scale_dense, int32_t *n_dense)
{
    if (n < 0 || npix < 0 || K < 1 || nthreads < 1 || (C < 0)) return OR_ERR_ARG;
    render_job_t base;
    memset(&base, 0, sizeof(base));
    base.n = n; base.mean2d = mean2d; base.conic = conic; base.depth = depth;
    base.alpha = alpha; base.valid = valid; base.feat = feat; base.C = C;
    base.K = K; base.alpha_min = alpha_min; base.alpha_max = alpha_max; base.T_min = T_min;
    base.tie_eps = tie_eps; base.npix = npix; base.pix = pix;
    base.out_q = out_q; base.ids = ids; base.wq = wq; base.cnt = cnt; base.tq = tq;
    base.out_dense = out_dense; base.t_final = t_final; base.n_members = n_members;
    base.n_proc = n_proc; base.tie = tie;
    base.members = members; base.max_members = members ? max_members : 0;
    base.scale_q = scale_q; base.scale_dense = scale_dense; base.n_dense = n_dense;
    base.nthreads = nthreads;
    render_job_t *jobs = (render_job_t *)calloc((size_t)nthreads, sizeof(render_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return OR_ERR_NOMEM; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base; jobs[t].tid = t;
        if (t > 0) pthread_create(&th[t], NULL, render_worker, &jobs[t]);
    }
    render_worker(&jobs[0]);
    int st = jobs[0].status;
    for (int t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) st = jobs[t].status;
    }
    free(jobs); free(th);
    return st;
}

/*
 * The near-tie classification of one pixel under a select rule of
 * or_render_rule, from its candidates as in or_classify_candidates.  Returns
 * the flags (or -1); kept [K] (nullable) receives the kept ids in depth order
 * (-1 padded) and tau [K] (nullable) the stratified boundaries.
 */
int or_classify_rule_candidates(int64_t n, const double *depth, const int64_t *id, const double *g,
                                const double *qabs, int rule, int K, double alpha_min,
                                double alpha_max, double T_min, double tie_eps, int64_t *kept,
                                double *tau)
{
    if (n < 0 || K < 1 || !depth || !id || !g || !qabs ||
        (rule != RULE_TOPK && rule != RULE_STRATIFIED && rule != RULE_RIEMANN))
        return -1;
    render_job_t J;
    memset(&J, 0, sizeof(J));
    int32_t tie = 0, cnt = 0;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    double *tv = (double *)malloc(sizeof(double) * (size_t)K);
    J.K = K; J.alpha_min = alpha_min; J.alpha_max = alpha_max; J.T_min = T_min;
    J.tie_eps = tie_eps; J.tie = &tie; J.cnt = &cnt; J.ids = ids; J.tau_out = tv; J.rule = rule;
    scratch_t S;
    memset(&S, 0, sizeof(S));
    int flags = -1;
    if (!ids || !tv) goto done;
    for (int64_t c = 0; c < n; ++c)
        if (add_candidate(&J, &S, depth[c], id[c], g[c], 1.0, 0.0, 0.0, qabs[c])) goto done;
    if (finish_list(&S) || render_rule_pixel(&J, &S, 0)) goto done;
    flags = tie;
    for (int k = 0; k < K; ++k) {
        if (kept) kept[k] = ids[k];
        if (tau) tau[k] = tv[k];
    }
done:
    free(S.m); free(S.border); free(S.a); free(S.w); free(S.wd); free(S.sel);
    free(ids); free(tv);
    return flags;
}

/*
 * Render the listed pixels with another select rule in place of Algorithm 1:
 * rule 1 = top-K (or_topk_list), rule 2 = Stratified-K (or_stratified_list),
 * rule 3 = Algorithm 1's selection with the Riemann weights of App. C
 * (or_riemann_list).
 * Outputs as or_render's Q-Render outputs (nullable): out [npix][C] (the kept
 * Gaussians' features with the rule's normalised weights), ids / wq [npix][K]
 * (depth order, -1 / 0 padded), cnt, n_members, n_proc (entries visited),
 * tie (classify_rule_ties), scale [npix] (sum |w| max|f|), tau [npix][K]
 * (stratified boundaries).
 */
int or_render_rule(int64_t n, const double *mean2d, const double *conic, const double *depth,
                   const double *alpha, const int32_t *valid, const double *feat, int C, int rule,
                   int K, double alpha_min, double alpha_max, double T_min, double tie_eps,
                   int64_t npix, const int32_t *pix, int nthreads, double *out, int32_t *ids,
                   double *wq, int32_t *cnt, int32_t *n_members, int32_t *n_proc, int32_t *tie,
                   double *scale, double *tau)
{
    if (n < 0 || npix < 0 || K < 1 || nthreads < 1 || C < 0 ||
        (rule != RULE_TOPK && rule != RULE_STRATIFIED && rule != RULE_RIEMANN))
        return OR_ERR_ARG;
    render_job_t base;
    memset(&base, 0, sizeof(base));
    base.n = n; base.mean2d = mean2d; base.conic = conic; base.depth = depth;
    base.alpha = alpha; base.valid = valid; base.feat = feat; base.C = C;
    base.K = K; base.alpha_min = alpha_min; base.alpha_max = alpha_max; base.T_min = T_min;
    base.tie_eps = tie_eps; base.npix = npix; base.pix = pix;
    base.out_q = out; base.ids = ids; base.wq = wq; base.cnt = cnt;
    base.n_members = n_members; base.n_proc = n_proc; base.tie = tie; base.scale_q = scale;
    base.rule = rule; base.tau_out = tau; base.nthreads = nthreads;
    render_job_t *jobs = (render_job_t *)calloc((size_t)nthreads, sizeof(render_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return OR_ERR_NOMEM; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base; jobs[t].tid = t;
        if (t > 0) pthread_create(&th[t], NULL, render_rule_worker, &jobs[t]);
    }
    render_rule_worker(&jobs[0]);
    int st = jobs[0].status;
    for (int t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) st = jobs[t].status;
    }
    free(jobs); free(th);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Backward of Algorithm 1 (the paper gives no formula; our derivation).      */
/* ------------------------------------------------------------------------ */
/*
 * For the quantile Gaussians j = 1..m of a pixel with a_j = alpha'_j,
 * P_j = prod_{l<j} (1 - a_l), T^Q = P_{m+1}, D = 1 - T^Q and
 * F = sum_j a_j P_j f_j / D, given g = dL/dF:
 *   dL/df_j = (a_j P_j / D) g
 *   dL/da_j = [P_j s_j - (1-a_j)^{-1} sum_{l>j} a_l P_l s_l] / D
 *             - (g.F) T^Q / ((1-a_j) D),          s_l = g . f_l
 * and through a = alpha * exp(-q/2) (zero where alpha*G >= alpha_max):
 *   dL/dalpha = dL/da * G,
 *   dL/d(A00, A01, A11) = dL/da * (-a/2) * (dx^2, 2 dx dy, dy^2).
 * The selection is piecewise constant in the inputs and is held fixed, so
 * non-selected Gaussians receive zero gradient.  Accumulation is serial and
 * in pixel order.  grad_feat [n][C], grad_alpha [n], grad_conic [n][3] are
 * accumulated into (the caller zeroes them).
 * The optional scale_feat [n], scale_alpha [n] and scale_conic [n][3]
 * accumulate, per Gaussian, the magnitudes of the parts its gradient is summed
 * from: |w_j| max_c |g_c| for a feature row, and for dL/da_j the same formula
 * with every part taken by magnitude (s_l -> sum_c |g_c f_lc|, g.F ->
 * sum_c |g_c| sum_l w_l |f_lc|) -- the size the sum could reach without
 * cancellation, against which the rounding error of a computed gradient is
 * measured.
 */
int or_backward(int64_t n, const double *mean2d, const double *conic, const double *depth,
                const double *alpha, const int32_t *valid, const double *feat, int C,
                int K, double alpha_min, double alpha_max,
                int64_t npix, const int32_t *pix, const double *grad_out,
                double *grad_feat, double *grad_alpha, double *grad_conic,
                double *scale_feat, double *scale_alpha, double *scale_conic)
{
    if (n < 0 || npix < 0 || K < 1 || C < 1 || !feat || !grad_out) return OR_ERR_ARG;
    render_job_t J;
    memset(&J, 0, sizeof(J));
    J.n = n; J.mean2d = mean2d; J.conic = conic; J.depth = depth; J.alpha = alpha;
    J.valid = valid; J.feat = feat; J.C = C; J.K = K; J.alpha_min = alpha_min;
    J.alpha_max = alpha_max; J.nthreads = 1;
    scratch_t S;
    memset(&S, 0, sizeof(S));
    int64_t *sid = NULL; double *sa = NULL, *sP = NULL, *ss = NULL, *F = NULL;
    double *sabs = NULL, *Fabs = NULL;
    int rc = OR_OK;
    sid = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    sa = (double *)malloc(sizeof(double) * (size_t)K);
    sP = (double *)malloc(sizeof(double) * (size_t)(K + 1));
    ss = (double *)malloc(sizeof(double) * (size_t)K);
    sabs = (double *)malloc(sizeof(double) * (size_t)K);
    F = (double *)malloc(sizeof(double) * (size_t)C);
    Fabs = (double *)malloc(sizeof(double) * (size_t)C);
    if (!sid || !sa || !sP || !ss || !sabs || !F || !Fabs) { rc = OR_ERR_NOMEM; goto done; }
    for (int64_t p = 0; p < npix; ++p) {
        int px = pix[2 * p], py = pix[2 * p + 1];
        if (build_list(&J, &S, px, py)) { rc = OR_ERR_NOMEM; goto done; }
        double Tq = 1.0; int64_t nproc = 0;
        int m = or_qrender_list(S.len, S.a, K, S.sel, S.w, &Tq, &nproc);
        if (m == 0) continue;
        int j = 0;
        for (int64_t i = 0; i < S.len; ++i)
            if (S.sel[i]) { sid[j] = i; sa[j] = S.a[i]; ++j; }
        sP[0] = 1.0;
        for (j = 0; j < m; ++j) sP[j + 1] = sP[j] * (1.0 - sa[j]);
        double D = 1.0 - sP[m];
        const double *g = grad_out + p * C;
        for (int c = 0; c < C; ++c) { F[c] = 0.0; Fabs[c] = 0.0; }
        for (j = 0; j < m; ++j) {
            const double *f = feat + S.m[sid[j]].id * C;
            double sj = 0.0, sjabs = 0.0;
            for (int c = 0; c < C; ++c) {
                sj += g[c] * f[c];
                sjabs += fabs(g[c] * f[c]);
                F[c] += sa[j] * sP[j] * f[c] / D;
                Fabs[c] += sa[j] * sP[j] * fabs(f[c]) / D;
            }
            ss[j] = sj;
            sabs[j] = sjabs;
        }
        double gF = 0.0, gFabs = 0.0;
        for (int c = 0; c < C; ++c) { gF += g[c] * F[c]; gFabs += fabs(g[c]) * Fabs[c]; }
        for (j = 0; j < m; ++j) {
            const member_t *mm = &S.m[sid[j]];
            double wj = sa[j] * sP[j] / D;
            double *gf = grad_feat + mm->id * C;
            for (int c = 0; c < C; ++c) gf[c] += wj * g[c];
            if (scale_feat) {
                double gmax = 0.0;
                for (int c = 0; c < C; ++c) gmax = fabs(g[c]) > gmax ? fabs(g[c]) : gmax;
                scale_feat[mm->id] += fabs(wj) * gmax;
            }
            double tail = 0.0, tailabs = 0.0;
            for (int l = j + 1; l < m; ++l) {
                tail += sa[l] * sP[l] * ss[l];
                tailabs += sa[l] * sP[l] * sabs[l];
            }
            double da = (sP[j] * ss[j] - tail / (1.0 - sa[j])) / D
                        - gF * sP[m] / ((1.0 - sa[j]) * D);
            double damag = (sP[j] * sabs[j] + tailabs / (1.0 - sa[j])) / D
                           + gFabs * sP[m] / ((1.0 - sa[j]) * D);
            if (mm->g < alpha_max) {
                if (grad_alpha) grad_alpha[mm->id] += da * mm->G;
                if (scale_alpha) scale_alpha[mm->id] += damag * mm->G;
                double h = -0.5 * sa[j] * da, hmag = 0.5 * sa[j] * damag;
                if (grad_conic) {
                    grad_conic[3 * mm->id] += h * mm->dx * mm->dx;
                    grad_conic[3 * mm->id + 1] += h * 2.0 * mm->dx * mm->dy;
                    grad_conic[3 * mm->id + 2] += h * mm->dy * mm->dy;
                }
                if (scale_conic) {
                    scale_conic[3 * mm->id] += hmag * mm->dx * mm->dx;
                    scale_conic[3 * mm->id + 1] += hmag * 2.0 * fabs(mm->dx * mm->dy);
                    scale_conic[3 * mm->id + 2] += hmag * mm->dy * mm->dy;
                }
            }
        }
    }
done:
    free(S.m); free(S.border); free(S.a); free(S.w); free(S.wd); free(S.sel);
    free(sid); free(sa); free(sP); free(ss); free(sabs); free(F); free(Fabs);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Storage formats of the feature table (not in the paper).                  */
/* ------------------------------------------------------------------------ */
static uint32_t f32_bits(float x) { uint32_t b; memcpy(&b, &x, 4); return b; }
static float bits_f32(uint32_t b) { float x; memcpy(&x, &b, 4); return x; }

/* BF16: the top 16 bits of the FP32 pattern, rounded to nearest, ties to even. */
void or_bf16_encode(const float *x, int64_t n, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t b = f32_bits(x[i]);
        if ((b & 0x7fffffffu) > 0x7f800000u) { out[i] = (uint16_t)((b >> 16) | 0x0040u); continue; }
        uint32_t lsb = (b >> 16) & 1u;
        out[i] = (uint16_t)((b + 0x7fffu + lsb) >> 16);
    }
}

void or_bf16_decode(const uint16_t *h, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = (double)bits_f32((uint32_t)h[i] << 16);
}

/*
 * FP8 E4M3 ("FN" variant): 1 sign, 4 exponent (bias 7), 3 mantissa bits; no
 * infinities; S.1111.111 is NaN, so the largest finite magnitude is
 * 1.75 * 2^8 = 448.  Exponent field 0 holds the subnormals m * 2^-9.
 */
double or_fp8_decode_one(uint8_t v)
{
    int s = v >> 7, e = (v >> 3) & 15, m = v & 7;
    if (e == 15 && m == 7) return NAN;
    double mag = (e == 0) ? ldexp((double)m, -9) : ldexp(1.0 + m / 8.0, e - 7);
    return s ? -mag : mag;
}

/* Round to the nearest finite E4M3 value, ties to the even code; saturate
 * magnitudes beyond 448 (and infinities) to 448; NaN stays NaN. */
uint8_t or_fp8_encode_one(float xf)
{
    double x = xf;
    if (x != x) return 0x7f;
    uint8_t sign = (f32_bits(xf) >> 31) ? 0x80 : 0x00;
    double a = fabs(x);
    if (a >= 448.0) return sign | 0x7e;
    /* codes 0..126 are the finite non-negative values in increasing order */
    int lo = 0, hi = 126;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (or_fp8_decode_one((uint8_t)mid) <= a) lo = mid; else hi = mid;
    }
    double vlo = or_fp8_decode_one((uint8_t)lo), vhi = or_fp8_decode_one((uint8_t)hi);
    int code;
    if (a - vlo < vhi - a) code = lo;
    else if (a - vlo > vhi - a) code = hi;
    else code = (lo & 1) ? hi : lo;
    return sign | (uint8_t)code;
}

void or_fp8_encode(const float *x, int64_t n, uint8_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_fp8_encode_one(x[i]);
}

void or_fp8_decode(const uint8_t *v, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_fp8_decode_one(v[i]);
}

/*
 * Per-row FP8 quantisation: scale_i = max_c |f_ic| / 448 in FP32 (1 for an
 * all-zero row), code_ic = E4M3(f_ic / scale_i) with the division in FP32.
 * The decoded value is E4M3^{-1}(code) * scale_i.
 */
void or_fp8_quantize_rows(const float *f, int64_t n, int C, uint8_t *codes, float *scale)
{
    for (int64_t i = 0; i < n; ++i) {
        float mx = 0.0f;
        for (int c = 0; c < C; ++c) { float v = fabsf(f[i * C + c]); if (v > mx) mx = v; }
        float s = mx > 0.0f ? mx / 448.0f : 1.0f;
        scale[i] = s;
        for (int c = 0; c < C; ++c) {
            volatile float r = f[i * C + c] / s;
            codes[i * C + c] = or_fp8_encode_one(r);
        }
    }
}
