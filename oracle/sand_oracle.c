/*
 * FP64 CPU oracle for the SAND query path — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  It shares no code, header or
 * table with the CUDA library; both read the same generated inputs.
 *
 * What it computes (SAND, arxiv 2604.25936):
 *   - Octree lookup (Sec. 3.2, Sec. 3.4, Eq. 7): descend a pointer octree over
 *     [-1,1]^3 from the root, choosing at every node the child octant by
 *     comparing each coordinate with the cell midpoint (a coordinate equal to
 *     the midpoint goes to the upper child), until a leaf.  The leaf gives the
 *     exit layer d (0..L) and, for d = 0, the stored SDF value at the leaf
 *     centre.  Level of detail (Sec. 3.4): d <- min(d, max_depth) when d > 0
 *     and max_depth > 0.  A NaN coordinate yields exit layer -1 and NaN.
 *   - T-MLP (Eq. 2): h_0 = x (or Fourier features of x), h_i = act(W_i h_{i-1}
 *     + b_i) with act = sin(omega0 * .) (SIREN), max(0, .) (ReLU) or
 *     sin(omega0 (|.| + 1) .) (FINER, the variable-periodic sine of the
 *     SAND-FINER backbone; SAND cites FINER without restating its formula, so
 *     this follows FINER's own definition, and its tests pin it to that
 *     definition evaluated in 50-digit arithmetic on hand-set layers),
 *     t_i = a_i . h_i + c_i, and for multiplicative tails (Eq. 3) with i >= 2
 *     t_i = (a_i . h_i + c_i) (b_i . h_i + e_i); y_i = y_{i-1} + t_i, y_0 = 0.
 *     The result for exit layer d is y_d.
 *   - Input gradient of y_d by reverse-mode chain rule, in double.
 * Everything is evaluated per point in double from the float32 master
 * parameters widened exactly; there is no blocking or reordering.
 *
 * Parameter block (float32, row-major, in this order):
 *   enc_B [m,3] (Fourier encoder only), W1 [W,D], b1 [W], Wh [L-1,W,W],
 *   bh [L-1,W], tail_w [L,2,W], tail_b [L,2].
 * Fourier features: gamma(x) = [sin(2 pi B_k . x) for k < m, cos(2 pi B_k . x) for k < m].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_TAIL_MULT 1
#define ORACLE_ACT_RELU 1
#define ORACLE_ACT_FINER 2
#define ORACLE_ENC_FOURIER 1

typedef struct {
    int L, W, D, tail_kind, act, enc, m;
    double omega0;
    const float *B, *W1, *b1, *Wh, *bh, *tw, *tb;
} model_t;

static int model_init(model_t *M, const int32_t *hdr, double omega0, const float *p) {
    M->L = hdr[0]; M->W = hdr[1]; M->D = hdr[2]; M->tail_kind = hdr[3];
    M->act = hdr[4]; M->enc = hdr[5]; M->m = hdr[6]; M->omega0 = omega0;
    if (M->L < 1 || M->W < 1 || M->D < 1) return -1;
    if (M->enc == ORACLE_ENC_FOURIER && M->D != 2 * M->m) return -1;
    if (M->enc != ORACLE_ENC_FOURIER && M->D != 3) return -1;
    const float *q = p;
    if (M->enc == ORACLE_ENC_FOURIER) { M->B = q; q += (size_t)M->m * 3; } else M->B = NULL;
    M->W1 = q; q += (size_t)M->W * M->D;
    M->b1 = q; q += M->W;
    M->Wh = q; q += (size_t)(M->L - 1) * M->W * M->W;
    M->bh = q; q += (size_t)(M->L - 1) * M->W;
    M->tw = q; q += (size_t)M->L * 2 * M->W;
    M->tb = q;
    return 0;
}

long long oracle_param_count(const int32_t *hdr) {
    long long L = hdr[0], W = hdr[1], D = hdr[2], m = hdr[6];
    long long n = W * D + W + (L - 1) * W * W + (L - 1) * W + L * 2 * W + L * 2;
    if (hdr[5] == ORACLE_ENC_FOURIER) n += m * 3;
    return n;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ lookup */
static int lookup_one(const int32_t *child, const uint8_t *depth, const float *far,
                      const float *x, int max_depth, double *far_out) {
    if (isnan(x[0]) || isnan(x[1]) || isnan(x[2])) { *far_out = NAN; return -1; }
    double lo[3] = {-1.0, -1.0, -1.0};
    double size = 2.0;
    int32_t node = 0;
    while (child[node] >= 0) {
        double half = size * 0.5;
        int oct = 0;
        for (int a = 0; a < 3; ++a) {
            double mid = lo[a] + half;
            if ((double)x[a] >= mid) { oct |= 1 << a; lo[a] = mid; }
        }
        size = half;
        node = child[node] + oct;
    }
    int d = depth[node];
    *far_out = (double)far[node];
    if (d > 0 && max_depth > 0 && d > max_depth) d = max_depth;
    return d;
}

int oracle_lookup(int n_nodes, const int32_t *child, const uint8_t *depth, const float *far,
                  const float *pts, int64_t n, int max_depth, int32_t *d_out, double *far_out) {
    (void)n_nodes;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double f;
        d_out[i] = lookup_one(child, depth, far, pts + 3 * i, max_depth, &f);
        if (far_out) far_out[i] = f;
    }
    return 0;
}

/* ------------------------------------------------------------------ T-MLP */
/* Features h_0 of the input point (and, if J != NULL, their Jacobian J[D][3]). */
static void features(const model_t *M, const float *xf, double *h0, double *J) {
    double x[3] = {xf[0], xf[1], xf[2]};
    if (M->enc != ORACLE_ENC_FOURIER) {
        for (int a = 0; a < 3; ++a) h0[a] = x[a];
        if (J) for (int r = 0; r < 3; ++r) for (int a = 0; a < 3; ++a) J[r * 3 + a] = (r == a);
        return;
    }
    const double tau = 2.0 * M_PI;
    for (int k = 0; k < M->m; ++k) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (double)M->B[k * 3 + a] * x[a];
        h0[k] = sin(tau * s);
        h0[M->m + k] = cos(tau * s);
        if (J) for (int a = 0; a < 3; ++a) {
            J[k * 3 + a] = tau * (double)M->B[k * 3 + a] * cos(tau * s);
            J[(M->m + k) * 3 + a] = -tau * (double)M->B[k * 3 + a] * sin(tau * s);
        }
    }
}

static double dot_f(const float *w, const double *h, int n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += (double)w[k] * h[k];
    return s;
}

/* Evaluate one point to exit layer d >= 1.  ys[l-1] = y_l for l = 1..d when ys != NULL.
 * grad (3 doubles) = d y_d / d x when grad != NULL.  work: (2*d + 2) * W + D*4 doubles. */
static double eval_one(const model_t *M, const float *x, int d, double *ys, double *grad, double *work) {
    const int W = M->W, D = M->D;
    double *h0 = work;                  /* D */
    double *J = h0 + D;                 /* D*3 */
    double *U = J + 3 * D;              /* d*W pre-activations u_l = W_l h_{l-1} + b_l */
    double *H = U + (size_t)d * W;      /* d*W activations h_l */
    double *g = H + (size_t)d * W;      /* W */
    double *g2 = g + W;                 /* max(W, D) */
    features(M, x, h0, grad ? J : NULL);
    double y = 0.0;
    for (int l = 1; l <= d; ++l) {
        const double *hp = (l == 1) ? h0 : H + (size_t)(l - 2) * W;
        const int fan = (l == 1) ? D : W;
        const float *Wl = (l == 1) ? M->W1 : M->Wh + (size_t)(l - 2) * W * W;
        const float *bl = (l == 1) ? M->b1 : M->bh + (size_t)(l - 2) * W;
        double *u = U + (size_t)(l - 1) * W, *h = H + (size_t)(l - 1) * W;
        for (int j = 0; j < W; ++j) {
            u[j] = dot_f(Wl + (size_t)j * fan, hp, fan) + (double)bl[j];
            if (M->act == ORACLE_ACT_RELU) h[j] = u[j] > 0.0 ? u[j] : 0.0;
            else if (M->act == ORACLE_ACT_FINER) h[j] = sin(M->omega0 * (fabs(u[j]) + 1.0) * u[j]);
            else h[j] = sin(M->omega0 * u[j]);
        }
        const float *a = M->tw + (size_t)(l - 1) * 2 * W, *b = a + W;
        double t0 = dot_f(a, h, W) + (double)M->tb[(l - 1) * 2];
        double t = t0;
        if (M->tail_kind == ORACLE_TAIL_MULT && l >= 2)
            t = t0 * (dot_f(b, h, W) + (double)M->tb[(l - 1) * 2 + 1]);
        y += t;
        if (ys) ys[l - 1] = y;
    }
    if (grad) {
        /* g accumulates d y_d / d h_l, walking l = d .. 1. */
        for (int j = 0; j < W; ++j) g[j] = 0.0;
        for (int l = d; l >= 1; --l) {
            const double *h = H + (size_t)(l - 1) * W, *u = U + (size_t)(l - 1) * W;
            const float *a = M->tw + (size_t)(l - 1) * 2 * W, *b = a + W;
            if (M->tail_kind == ORACLE_TAIL_MULT && l >= 2) {
                double ta = dot_f(a, h, W) + (double)M->tb[(l - 1) * 2];
                double tb = dot_f(b, h, W) + (double)M->tb[(l - 1) * 2 + 1];
                for (int j = 0; j < W; ++j) g[j] += tb * (double)a[j] + ta * (double)b[j];
            } else {
                for (int j = 0; j < W; ++j) g[j] += (double)a[j];
            }
            for (int j = 0; j < W; ++j) {
                double dact;
                if (M->act == ORACLE_ACT_RELU) dact = u[j] > 0.0 ? 1.0 : 0.0;
                else if (M->act == ORACLE_ACT_FINER)  /* d/du sin(w0 (|u| + 1) u) */
                    dact = M->omega0 * (2.0 * fabs(u[j]) + 1.0) * cos(M->omega0 * (fabs(u[j]) + 1.0) * u[j]);
                else dact = M->omega0 * cos(M->omega0 * u[j]);
                g[j] *= dact;               /* now d y / d u_l */
            }
            const int fan = (l == 1) ? D : W;
            const float *Wl = (l == 1) ? M->W1 : M->Wh + (size_t)(l - 2) * W * W;
            for (int k = 0; k < fan; ++k) {
                double s = 0.0;
                for (int j = 0; j < W; ++j) s += (double)Wl[(size_t)j * fan + k] * g[j];
                g2[k] = s;                  /* d y / d h_{l-1} (partial, tails added next step) */
            }
            if (l > 1) memcpy(g, g2, sizeof(double) * W);
        }
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += g2[k] * J[k * 3 + a];
            grad[a] = s;
        }
    }
    return y;
}

static size_t work_doubles(const model_t *M) {
    return (size_t)M->D * 4 + (size_t)(2 * M->L + 2) * M->W + (M->W > M->D ? M->W : M->D) + 16;
}

/* Evaluate points at given exit layers (depth[i], or const_depth when depth == NULL).
 * Exit layers <= 0 give y = 0 and a zero gradient (the caller substitutes stored values).
 * y: [n]; grad: [n][3] or NULL; ys_all: [n][L] (cumulative outputs y_1..y_d, rest 0) or NULL. */
int oracle_eval(const int32_t *hdr, double omega0, const float *params, const float *pts, int64_t n,
                const int32_t *depth, int const_depth, double *y, double *grad, double *ys_all) {
    model_t M;
    if (model_init(&M, hdr, omega0, params)) return -1;
    int bad = 0;
    #pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * work_doubles(&M));
        double *ys = (double *)malloc(sizeof(double) * M.L);
        if (!work || !ys) { bad = 1; }
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            if (bad) continue;
            int d = depth ? depth[i] : const_depth;
            if (d > M.L) d = M.L;
            if (d <= 0) {
                y[i] = 0.0;
                if (grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = 0.0;
                if (ys_all) for (int l = 0; l < M.L; ++l) ys_all[i * M.L + l] = 0.0;
                continue;
            }
            y[i] = eval_one(&M, pts + 3 * i, d, ys, grad ? grad + 3 * i : NULL, work);
            if (ys_all) for (int l = 0; l < M.L; ++l) ys_all[i * M.L + l] = (l < d) ? ys[l] : 0.0;
        }
        free(work); free(ys);
    }
    return bad ? -2 : 0;
}

/* Smallest |u_l[j]| over the pre-activations of layers 1..d of each point (Eq. 1:
 * u_l = W_l h_{l-1} + b_l), +inf for d <= 0.  A ReLU network's gradient is discontinuous
 * where some u_l[j] = 0; two evaluations whose u differ by less than margin[i] take the
 * same ReLU decisions at point i. */
int oracle_preact_margin(const int32_t *hdr, double omega0, const float *params, const float *pts, int64_t n,
                         const int32_t *depth, int const_depth, double *margin) {
    model_t M;
    if (model_init(&M, hdr, omega0, params)) return -1;
    int bad = 0;
    #pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * work_doubles(&M));
        double *ys = (double *)malloc(sizeof(double) * M.L);
        if (!work || !ys) { bad = 1; }
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            if (bad) continue;
            int d = depth ? depth[i] : const_depth;
            if (d > M.L) d = M.L;
            margin[i] = INFINITY;
            if (d <= 0) continue;
            (void)eval_one(&M, pts + 3 * i, d, ys, NULL, work);
            const double *U = work + 4 * (size_t)M.D;  /* eval_one's layout: h0 [D], J [3D], U [d][W] */
            for (int64_t k = 0; k < (int64_t)d * M.W; ++k)
                if (fabs(U[k]) < margin[i]) margin[i] = fabs(U[k]);
        }
        free(work); free(ys);
    }
    return bad ? -2 : 0;
}

/* The SAND query (Sec. 3.4): lookup, then the stored value for exit layer 0,
 * NaN for a NaN point, else y_d.  d_out (nullable) receives the exit layers
 * (-1 for NaN points).  grad (nullable) = d y / d x (0 for exit layer 0). */
int oracle_query(const int32_t *hdr, double omega0, const float *params,
                 int n_nodes, const int32_t *child, const uint8_t *depth, const float *far,
                 const float *pts, int64_t n, int max_depth, double *y, double *grad, int32_t *d_out) {
    model_t M;
    if (model_init(&M, hdr, omega0, params)) return -1;
    (void)n_nodes;
    int bad = 0;
    #pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * work_doubles(&M));
        if (!work) bad = 1;
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            if (bad) continue;
            double f;
            int d = lookup_one(child, depth, far, pts + 3 * i, max_depth, &f);
            if (d_out) d_out[i] = d;
            if (d > M.L) d = M.L;
            if (d <= 0) {
                y[i] = f;   /* stored far value, or NaN for a NaN point */
                if (grad) {
                    double gv = (d < 0) ? NAN : 0.0;
                    grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = gv;
                }
                continue;
            }
            y[i] = eval_one(&M, pts + 3 * i, d, NULL, grad ? grad + 3 * i : NULL, work);
        }
        free(work);
    }
    return bad ? -2 : 0;
}

/* ------------------------------------------------------------------ training loss and gradient
 * The T-MLP training objective (Sec. 3.3, Eq. 4 with the L1 SDF loss of Eq. 8):
 *     L = sum_{i=1..L} (1/n) sum_x | y_i(x) - y_gt(x) |,
 * y_i the cumulative output up to tail i (Eq. 2 / Eq. 3).  Its gradient with respect to every
 * trained parameter (W_l, b_l, tail weights and biases; a Fourier matrix B is fixed, gradient
 * 0) by reverse-mode chain rule, per point in double, summed over the points.  The derivative
 * of |r| is taken as sign(r) with sign(0) = 0.
 * With G_k = (1/n) sum_{i>=k} sign(y_i - y_gt) = dL/dt_k (y_i = t_1 + ... + t_i), walking
 * l = L .. 1 with g = dL/dh_l (0 above layer L):
 *   linear tail:  dL/da_l += G_l h_l,  dL/dc_l += G_l,  g += G_l a_l;
 *   mult. tail:   t_l = ta tb with ta = a.h + c, tb = b.h + e:  dL/da += G tb h, dL/dc += G tb,
 *                 dL/db += G ta h, dL/de += G ta, g += G (tb a + ta b);
 *   delta = g * act'(u_l);  dL/db_l += delta;  dL/dW_l += delta h_{l-1}^T;  g <- W_l^T delta.
 * loss: [1]; grad: [n_params] in the parameter-block layout.  Each thread sums its points into
 * its own block; the blocks are added in thread order. */
static double act_slope(const model_t *M, double u) {
    if (M->act == ORACLE_ACT_RELU) return u > 0.0 ? 1.0 : 0.0;
    if (M->act == ORACLE_ACT_FINER) return M->omega0 * (2.0 * fabs(u) + 1.0) * cos(M->omega0 * (fabs(u) + 1.0) * u);
    return M->omega0 * cos(M->omega0 * u);
}

static double act_value(const model_t *M, double u) {
    if (M->act == ORACLE_ACT_RELU) return u > 0.0 ? u : 0.0;
    if (M->act == ORACLE_ACT_FINER) return sin(M->omega0 * (fabs(u) + 1.0) * u);
    return sin(M->omega0 * u);
}

int oracle_train_grad(const int32_t *hdr, double omega0, const float *params, const float *pts,
                      const float *gt, int64_t n, double *loss, double *grad) {
    model_t M;
    if (model_init(&M, hdr, omega0, params)) return -1;
    if (n <= 0) return -3;
    const int L = M.L, W = M.W, D = M.D;
    const long long np = oracle_param_count(hdr);
    /* offsets of the parameter groups in the block */
    const size_t oB = 0, oW1 = (M.enc == ORACLE_ENC_FOURIER) ? (size_t)M.m * 3 : 0;
    const size_t ob1 = oW1 + (size_t)W * D, oWh = ob1 + W, obh = oWh + (size_t)(L - 1) * W * W;
    const size_t otw = obh + (size_t)(L - 1) * W, otb = otw + (size_t)L * 2 * W;
    (void)oB;
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nt * (size_t)np, sizeof(double));
    double *lacc = (double *)calloc((size_t)nt, sizeof(double));
    if (!acc || !lacc) { free(acc); free(lacc); return -2; }
    int bad = 0;
    #pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *G = acc + (size_t)tid * (size_t)np;
        double *h0 = (double *)malloc(sizeof(double) * D);
        double *U = (double *)malloc(sizeof(double) * (size_t)L * W);
        double *H = (double *)malloc(sizeof(double) * (size_t)L * W);
        double *TA = (double *)malloc(sizeof(double) * L);
        double *TB = (double *)malloc(sizeof(double) * L);
        double *Y = (double *)malloc(sizeof(double) * L);
        double *Gt = (double *)malloc(sizeof(double) * L);
        double *g = (double *)malloc(sizeof(double) * W);
        double *dl = (double *)malloc(sizeof(double) * W);
        if (!h0 || !U || !H || !TA || !TB || !Y || !Gt || !g || !dl) bad = 1;
        #pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            if (bad) continue;
            features(&M, pts + 3 * i, h0, NULL);
            double y = 0.0;
            for (int l = 1; l <= L; ++l) {
                const double *hp = (l == 1) ? h0 : H + (size_t)(l - 2) * W;
                const int fan = (l == 1) ? D : W;
                const float *Wl = (l == 1) ? M.W1 : M.Wh + (size_t)(l - 2) * W * W;
                const float *bl = (l == 1) ? M.b1 : M.bh + (size_t)(l - 2) * W;
                double *u = U + (size_t)(l - 1) * W, *h = H + (size_t)(l - 1) * W;
                for (int j = 0; j < W; ++j) {
                    u[j] = dot_f(Wl + (size_t)j * fan, hp, fan) + (double)bl[j];
                    h[j] = act_value(&M, u[j]);
                }
                const float *a = M.tw + (size_t)(l - 1) * 2 * W, *b = a + W;
                TA[l - 1] = dot_f(a, h, W) + (double)M.tb[(l - 1) * 2];
                TB[l - 1] = (M.tail_kind == ORACLE_TAIL_MULT && l >= 2) ? dot_f(b, h, W) + (double)M.tb[(l - 1) * 2 + 1] : 1.0;
                y += TA[l - 1] * TB[l - 1];
                Y[l - 1] = y;
            }
            const double target = (double)gt[i];
            double s = 0.0;
            for (int l = L; l >= 1; --l) {
                const double r = Y[l - 1] - target;
                lacc[tid] += fabs(r);
                s += (r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0)) / (double)n;
                Gt[l - 1] = s;
            }
            for (int j = 0; j < W; ++j) g[j] = 0.0;
            for (int l = L; l >= 1; --l) {
                const double *h = H + (size_t)(l - 1) * W, *u = U + (size_t)(l - 1) * W;
                const float *a = M.tw + (size_t)(l - 1) * 2 * W, *b = a + W;
                double *da = G + otw + (size_t)(l - 1) * 2 * W, *db = da + W;
                double *dc = G + otb + (size_t)(l - 1) * 2;
                const double Gl = Gt[l - 1];
                if (M.tail_kind == ORACLE_TAIL_MULT && l >= 2) {
                    for (int j = 0; j < W; ++j) {
                        da[j] += Gl * TB[l - 1] * h[j];
                        db[j] += Gl * TA[l - 1] * h[j];
                        g[j] += Gl * (TB[l - 1] * (double)a[j] + TA[l - 1] * (double)b[j]);
                    }
                    dc[0] += Gl * TB[l - 1];
                    dc[1] += Gl * TA[l - 1];
                } else {
                    for (int j = 0; j < W; ++j) {
                        da[j] += Gl * h[j];
                        g[j] += Gl * (double)a[j];
                    }
                    dc[0] += Gl;
                }
                for (int j = 0; j < W; ++j) dl[j] = g[j] * act_slope(&M, u[j]);
                const int fan = (l == 1) ? D : W;
                const double *hp = (l == 1) ? h0 : H + (size_t)(l - 2) * W;
                const float *Wl = (l == 1) ? M.W1 : M.Wh + (size_t)(l - 2) * W * W;
                double *dW = G + ((l == 1) ? oW1 : oWh + (size_t)(l - 2) * W * W);
                double *dbias = G + ((l == 1) ? ob1 : obh + (size_t)(l - 2) * W);
                for (int j = 0; j < W; ++j) {
                    dbias[j] += dl[j];
                    for (int k = 0; k < fan; ++k) dW[(size_t)j * fan + k] += dl[j] * hp[k];
                }
                if (l > 1) {
                    for (int k = 0; k < W; ++k) {
                        double t = 0.0;
                        for (int j = 0; j < W; ++j) t += (double)Wl[(size_t)j * W + k] * dl[j];
                        g[k] = t;
                    }
                }
            }
        }
        free(h0); free(U); free(H); free(TA); free(TB); free(Y); free(Gt); free(g); free(dl);
    }
    if (!bad) {
        double ls = 0.0;
        for (int t = 0; t < nt; ++t) ls += lacc[t];
        *loss = ls / (double)n;
        for (long long k = 0; k < np; ++k) {
            double s = 0.0;
            for (int t = 0; t < nt; ++t) s += acc[(size_t)t * (size_t)np + (size_t)k];
            grad[k] = s;
        }
    }
    free(acc);
    free(lacc);
    return bad ? -2 : 0;
}
