/*
 * oracle.c -- plain FP64 CPU oracle for the H-HIGNN mobility product.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * helper with the CUDA library, and it is compiled with
 * -O2 -ffp-contract=off -fno-fast-math so that every floating-point
 * operation is a single correctly rounded IEEE operation in source order.
 *
 * What it computes (H-HIGNN, arXiv 2505.08174):
 *   - the pair kernel M_ij = S(MLP(f)) / |r| with r = x_i - x_j and
 *     f = [r/|r|, a/|r|]  (Section 2.3, Eq. 4), or the closed-form
 *     Rotne-Prager-Yamakawa tensor;
 *   - the single-body mobility alpha_1 = I / (6 pi mu a)  (Section 2.2, Eq. 2);
 *   - the exact dense product U = alpha_1 F + sum_{j != i} M_ij F_j
 *     (Eq. 6 restricted to M^(1) + M^(t,2));
 *   - the cluster tree (Definition 1, Section 3.1) by Morton bisection;
 *   - BuildPartition (Algorithm 1) with the admissibility test of Eq. 7 on
 *     bounding boxes;
 *   - block ACA with 3x3 elements (Algorithm 2, Eqs. 8-10);
 *   - the H-matrix product built from the above;
 *   - the relative error of Eq. 11;
 *   - the analytic gradient of L = sum_i w_i . U_i w.r.t. F, X and theta,
 *     and the training loss of Eq. 5 with its gradient and an Adam step;
 *   - the short-range terms M^(s,2), M^(t,3), M^(s,3) of Eq. 6 (Eq. 2 with
 *     the Eq. 4 normalisations) over neighbours within R_cut;
 *   - the bead forces of the filament suspension (bond, bending, gravity;
 *     Section 4.3), which the explicit Euler step x <- x + dt U(x, F(x)) of
 *     Section 2.5 uses.
 *
 * Readings of points the paper leaves open are stated where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Pair kernel                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int kind;            /* 0 = MLP, 1 = RPY */
    int width;           /* hidden width of the MLP (depth is fixed at 3) */
    const double *theta; /* packed parameters: per layer W[out,in] then b[out] */
    double a;            /* particle radius */
    double mu;           /* viscosity */
} or_kernel;

static double or_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }
static double or_silu(double x) { return x / (1.0 + exp(-x)); }

/* One dense layer y = W x + b with W [n_out, n_in] row-major. */
static const double *or_layer(const double *p, int n_in, int n_out, const double *x, double *y)
{
    const double *W = p, *b = p + (size_t)n_in * n_out;
    for (int o = 0; o < n_out; ++o) {
        double s = 0.0;
        for (int i = 0; i < n_in; ++i) s += W[(size_t)o * n_in + i] * x[i];
        y[o] = s + b[o];
    }
    return b + n_out;
}

/* MLP 4 -> w -> w -> w -> 6 with SiLU after each hidden layer, linear output.
 * z[3][w] receives the hidden pre-activations (may be NULL). */
static void or_mlp_fwd(const double *theta, int w, const double f[4], double o[6], double *z)
{
    double h[256], g[256];
    const double *p = theta;
    p = or_layer(p, 4, w, f, h);
    if (z) memcpy(z, h, sizeof(double) * w);
    for (int i = 0; i < w; ++i) h[i] = or_silu(h[i]);
    p = or_layer(p, w, w, h, g);
    if (z) memcpy(z + w, g, sizeof(double) * w);
    for (int i = 0; i < w; ++i) g[i] = or_silu(g[i]);
    p = or_layer(p, w, w, g, h);
    if (z) memcpy(z + 2 * w, h, sizeof(double) * w);
    for (int i = 0; i < w; ++i) h[i] = or_silu(h[i]);
    or_layer(p, w, 6, h, o);
}

void or_mlp_forward(const double *theta, int w, const double f[4], double o[6]) { or_mlp_fwd(theta, w, f, o, NULL); }

/* Reverse pass of the MLP for output cotangent go[6]: gf[4] receives dL/df
 * and gtheta (same packing as theta, may be NULL) is incremented. */
static void or_mlp_bwd(const double *theta, int w, const double f[4], const double go[6], double gf[4],
                       double *gtheta)
{
    double z[768], h0[4], h1[256], h2[256], h3[256], o[6];
    or_mlp_fwd(theta, w, f, o, z);
    memcpy(h0, f, sizeof h0);
    for (int i = 0; i < w; ++i) {
        h1[i] = or_silu(z[i]);
        h2[i] = or_silu(z[w + i]);
        h3[i] = or_silu(z[2 * w + i]);
    }
    const int dims[5] = {4, w, w, w, 6};
    size_t off[4], cur = 0;
    for (int l = 0; l < 4; ++l) { off[l] = cur; cur += (size_t)dims[l] * dims[l + 1] + dims[l + 1]; }
    const double *acts[4] = {h0, h1, h2, h3};
    double gcur[256], gprev[256];
    memcpy(gcur, go, sizeof(double) * 6);
    for (int l = 3; l >= 0; --l) {
        int ni = dims[l], no = dims[l + 1];
        const double *W = theta + off[l];
        /* gcur is dL/d(pre-activation output of layer l) */
        if (gtheta) {
            double *gW = gtheta + off[l], *gb = gW + (size_t)ni * no;
            for (int oo = 0; oo < no; ++oo) {
                for (int i = 0; i < ni; ++i) gW[(size_t)oo * ni + i] += gcur[oo] * acts[l][i];
                gb[oo] += gcur[oo];
            }
        }
        for (int i = 0; i < ni; ++i) {
            double s = 0.0;
            for (int oo = 0; oo < no; ++oo) s += W[(size_t)oo * ni + i] * gcur[oo];
            gprev[i] = s;
        }
        if (l > 0) {
            /* through SiLU: d/dz [z sigma(z)] = sigma(z) (1 + z (1 - sigma(z))) */
            const double *zl = z + (size_t)(l - 1) * w;
            for (int i = 0; i < ni; ++i) {
                double sg = or_sigmoid(zl[i]);
                gcur[i] = gprev[i] * sg * (1.0 + zl[i] * (1.0 - sg));
            }
        } else {
            memcpy(gf, gprev, sizeof(double) * 4);
        }
    }
}

/* sym3x3: o -> [[o0,o3,o4],[o3,o1,o5],[o4,o5,o2]] (row-major 9). */
static void or_sym3(const double o[6], double S[9])
{
    S[0] = o[0]; S[1] = o[3]; S[2] = o[4];
    S[3] = o[3]; S[4] = o[1]; S[5] = o[5];
    S[6] = o[4]; S[7] = o[5]; S[8] = o[2];
}

/* 3x3 mobility block for separation r = x_target - x_source (r != 0). */
void or_pair_block(const or_kernel *k, const double r[3], double K[9])
{
    double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (k->kind == 0) {
        double f[4] = {r[0] / d, r[1] / d, r[2] / d, k->a / d}, o[6], S[9];
        or_mlp_fwd(k->theta, k->width, f, o, NULL);
        or_sym3(o, S);
        for (int e = 0; e < 9; ++e) K[e] = S[e] / d;
    } else {
        /* Rotne-Prager-Yamakawa, unbounded domain. */
        double a = k->a, A, B;
        if (d >= 2.0 * a) {
            double c = 1.0 / (8.0 * OR_PI * k->mu * d);
            A = c * (1.0 + 2.0 * a * a / (3.0 * d * d));
            B = c * (1.0 - 2.0 * a * a / (d * d));
        } else {
            double c = 1.0 / (6.0 * OR_PI * k->mu * a);
            A = c * (1.0 - 9.0 * d / (32.0 * a));
            B = c * (3.0 * d / (32.0 * a));
        }
        double u[3] = {r[0] / d, r[1] / d, r[2] / d};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) K[3 * i + j] = (i == j ? A : 0.0) + B * u[i] * u[j];
    }
}

/* alpha_1 = 1 / (6 pi mu a): the single-body mobility (scalar times I). */
double or_self_mobility(double a, double mu) { return 1.0 / (6.0 * OR_PI * mu * a); }

/* ------------------------------------------------------------------------ */
/* Exact dense product (ground truth for Eq. 11)                            */
/* ------------------------------------------------------------------------ */

/* U_row = alpha_1 F_i + sum_{j != i} K(x_i - x_j) F_j for the listed rows i.
 * rows == NULL means all n rows.  with_self == 0 leaves out alpha_1 (that is
 * M^(t,2) F, the quantity of Eq. 11). */
void or_dense_matvec(int n, const double *X, const double *F, const or_kernel *k, const int64_t *rows,
                     int64_t nrows, int with_self, double *U)
{
    double a1 = or_self_mobility(k->a, k->mu);
    if (!rows) nrows = n;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows ? rows[t] : t;
        double u[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3] = {X[3 * i] - X[3 * j], X[3 * i + 1] - X[3 * j + 1], X[3 * i + 2] - X[3 * j + 2]};
            double K[9];
            or_pair_block(k, r, K);
            for (int a = 0; a < 3; ++a)
                u[a] += K[3 * a] * F[3 * j] + K[3 * a + 1] * F[3 * j + 1] + K[3 * a + 2] * F[3 * j + 2];
        }
        for (int a = 0; a < 3; ++a) U[3 * t + a] = (with_self ? a1 * F[3 * i + a] : 0.0) + u[a];
    }
}

/* The same exact product for nf force vectors at once (F, U: [nf][n][3] and
 * [nf][nrows][3]); each pair block is evaluated once and applied to every
 * force vector, in the same order of j as or_dense_matvec. */
void or_dense_matvec_multi(int n, const double *X, int nf, const double *F, const or_kernel *k, const int64_t *rows,
                           int64_t nrows, int with_self, double *U)
{
    double a1 = or_self_mobility(k->a, k->mu);
    if (!rows) nrows = n;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows ? rows[t] : t;
        double u[8][3] = {{0}};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3] = {X[3 * i] - X[3 * j], X[3 * i + 1] - X[3 * j + 1], X[3 * i + 2] - X[3 * j + 2]};
            double K[9];
            or_pair_block(k, r, K);
            for (int f = 0; f < nf; ++f) {
                const double *Fj = F + 3 * ((size_t)f * n + j);
                for (int a = 0; a < 3; ++a) u[f][a] += K[3 * a] * Fj[0] + K[3 * a + 1] * Fj[1] + K[3 * a + 2] * Fj[2];
            }
        }
        for (int f = 0; f < nf; ++f)
            for (int a = 0; a < 3; ++a)
                U[3 * ((size_t)f * nrows + t) + a] = (with_self ? a1 * F[3 * ((size_t)f * n + i) + a] : 0.0) + u[f][a];
    }
}

/* Dense 3n x 3n matrix (row-major, element (3i+a, 3j+b)). */
void or_dense_matrix(int n, const double *X, const or_kernel *k, int with_self, double *M)
{
    double a1 = or_self_mobility(k->a, k->mu);
    size_t ld = 3 * (size_t)n;
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double K[9] = {0};
            if (i != j) {
                double r[3] = {X[3 * i] - X[3 * j], X[3 * i + 1] - X[3 * j + 1], X[3 * i + 2] - X[3 * j + 2]};
                or_pair_block(k, r, K);
            } else if (with_self) {
                K[0] = K[4] = K[8] = a1;
            }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[(3 * (size_t)i + a) * ld + 3 * (size_t)j + b] = K[3 * a + b];
        }
}

/* ------------------------------------------------------------------------ */
/* Analytic gradient of L = sum_i w_i . U_i (MLP kernel)                     */
/* ------------------------------------------------------------------------ */

/* For every pair i != j with r = x_i - x_j, d = |r|, f = [r/d, a/d]:
 *   L_ij = <w_i F_j^T, S(o(f))> / d.
 * dL/dF_j = alpha_1 w_j + sum_i K(x_i - x_j)^T w_i;
 * dL/do_c = <G, E_c> / d with G = w_i F_j^T and E_c the 0/1 pattern of o_c in S;
 * dL/dr   = -(<G,S>/d) r / d^2 + (I - r r^T/d^2) / d * g_f[0:3] - a r / d^3 * g_f[3];
 * dL/dx_i += dL/dr, dL/dx_j -= dL/dr; dL/dtheta by the MLP reverse pass.
 * Any output may be NULL.  gtheta is overwritten. */
void or_dense_grad(int n, const double *X, const double *F, const double *W, const or_kernel *k, int with_self,
                   double *gF, double *gX, double *gtheta)
{
    const int w = k->width;
    const size_t P = (size_t)(4 * w + w + 2 * (w * w + w) + 6 * w + 6);
    double a1 = or_self_mobility(k->a, k->mu);
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double *gXp = (double *)calloc((size_t)nt * 3 * n, sizeof(double));
    double *gTp = (double *)calloc((size_t)nt * P, sizeof(double));
    if (gF)
        for (int j = 0; j < n; ++j)
            for (int a = 0; a < 3; ++a) gF[3 * j + a] = with_self ? a1 * W[3 * j + a] : 0.0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < n; ++j) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *myX = gXp + (size_t)tid * 3 * n, *myT = gTp + (size_t)tid * P;
        double gfj[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i) {
            if (i == j) continue;
            double r[3] = {X[3 * i] - X[3 * j], X[3 * i + 1] - X[3 * j + 1], X[3 * i + 2] - X[3 * j + 2]};
            double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double f[4] = {r[0] / d, r[1] / d, r[2] / d, k->a / d}, o[6], S[9];
            or_mlp_fwd(k->theta, w, f, o, NULL);
            or_sym3(o, S);
            /* dF_j += K^T w_i = S w_i / d (S symmetric) */
            for (int a = 0; a < 3; ++a)
                gfj[a] += (S[3 * a] * W[3 * i] + S[3 * a + 1] * W[3 * i + 1] + S[3 * a + 2] * W[3 * i + 2]) / d;
            if (!gX && !gtheta) continue;
            double G[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) G[3 * a + b] = W[3 * i + a] * F[3 * j + b];
            double go[6] = {G[0] / d, G[4] / d, G[8] / d, (G[1] + G[3]) / d, (G[2] + G[6]) / d, (G[5] + G[7]) / d};
            double gf[4];
            or_mlp_bwd(k->theta, w, f, go, gf, gtheta ? myT : NULL);
            if (gX) {
                double gs = 0.0;
                for (int e = 0; e < 9; ++e) gs += G[e] * S[e];
                gs /= d;
                double rg = (r[0] * gf[0] + r[1] * gf[1] + r[2] * gf[2]) / d;
                for (int a = 0; a < 3; ++a) {
                    double g = -gs * r[a] / (d * d) + (gf[a] - rg * r[a] / d) / d - k->a * r[a] / (d * d * d) * gf[3];
                    myX[3 * i + a] += g;
                    myX[3 * j + a] -= g;
                }
            }
        }
        if (gF)
            for (int a = 0; a < 3; ++a) gF[3 * j + a] += gfj[a];
    }
    if (gX) {
        memset(gX, 0, sizeof(double) * 3 * n);
        for (int t = 0; t < nt; ++t)
            for (int i = 0; i < 3 * n; ++i) gX[i] += gXp[(size_t)t * 3 * n + i];
    }
    if (gtheta) {
        memset(gtheta, 0, sizeof(double) * P);
        for (int t = 0; t < nt; ++t)
            for (size_t i = 0; i < P; ++i) gtheta[i] += gTp[(size_t)t * P + i];
    }
    free(gXp);
    free(gTp);
}

/* ------------------------------------------------------------------------ */
/* Training of the pair MLP (Section 2.3, Eq. 5)                             */
/* ------------------------------------------------------------------------ */

/* Two-particle samples s: separation r_s (particle 1 minus particle 2), unit
 * force e_s on particle 2, teacher velocity of particle 1 U_s (3-vector).
 * The surrogate velocity is U^HIGNN = K(r_s) e_s (the alpha_1 term is zero
 * because particle 1 carries no force).
 * Loss (Eq. 5): L = (1/B) sum_s |U_s - K(r_s) e_s|^2 / |U_s|^2.
 * Returns L; gtheta (may be NULL) is overwritten with dL/dtheta. */
double or_train_loss_grad(const double *theta, int w, int64_t B, const double *r, const double *e, const double *U,
                          double a, double *gtheta)
{
    const size_t P = (size_t)(4 * w + w + 2 * (w * w + w) + 6 * w + 6);
    if (gtheta) memset(gtheta, 0, sizeof(double) * P);
    double L = 0.0;
    for (int64_t s = 0; s < B; ++s) {
        const double *rs = r + 3 * s, *es = e + 3 * s, *Us = U + 3 * s;
        double d = sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
        double f[4] = {rs[0] / d, rs[1] / d, rs[2] / d, a / d}, o[6], S[9];
        or_mlp_fwd(theta, w, f, o, NULL);
        or_sym3(o, S);
        double res[3], nU = Us[0] * Us[0] + Us[1] * Us[1] + Us[2] * Us[2];
        for (int i = 0; i < 3; ++i)
            res[i] = (S[3 * i] * es[0] + S[3 * i + 1] * es[1] + S[3 * i + 2] * es[2]) / d - Us[i];
        L += (res[0] * res[0] + res[1] * res[1] + res[2] * res[2]) / nU;
        if (gtheta) {
            /* dL/dKe = 2 res / (B |U|^2); K e = S e / d; dL/dS_ab = g_a e_b / d */
            double g[3], G[9];
            for (int i = 0; i < 3; ++i) g[i] = 2.0 * res[i] / ((double)B * nU);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) G[3 * i + j] = g[i] * es[j] / d;
            double go[6] = {G[0], G[4], G[8], G[1] + G[3], G[2] + G[6], G[5] + G[7]}, gf[4];
            or_mlp_bwd(theta, w, f, go, gf, gtheta);
        }
    }
    return L / (double)B;
}

/* One Adam step (Kingma & Ba 2015) with bias correction, step count t >= 1. */
void or_adam_step(double *theta, const double *g, double *m, double *v, int64_t P, double lr, double b1, double b2,
                  double eps, int t)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < P; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Morton order (cluster-tree geometry, Section 3.1)                         */
/* ------------------------------------------------------------------------ */

/* Reading of the bounding-box bisection: quantise every centre into the
 * global bounding cube on a 2^21 grid per axis and interleave the bits
 * x, y, z from the most significant down (x highest).  lo = per-axis
 * minimum, E = largest per-axis extent, s = 2^21 / E,
 * q = min(floor((x - lo) * s), 2^21 - 1). */
void or_morton_codes(int n, const double *X, uint64_t *codes)
{
    if (n <= 0) return;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = X[a]; hi[a] = X[a]; }
    for (int i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = X[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double E = 0.0;
    for (int a = 0; a < 3; ++a)
        if (hi[a] - lo[a] > E) E = hi[a] - lo[a];
    double s = E > 0.0 ? 2097152.0 / E : 0.0;
    for (int i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
            double t = floor((X[3 * i + a] - lo[a]) * s);
            q[a] = t > 2097151.0 ? 2097151u : (uint32_t)t;
        }
        uint64_t c = 0;
        for (int b = 20; b >= 0; --b)
            c = (c << 3) | ((uint64_t)((q[0] >> b) & 1u) << 2) | ((uint64_t)((q[1] >> b) & 1u) << 1) |
                (uint64_t)((q[2] >> b) & 1u);
        codes[i] = c;
    }
}

typedef struct { uint64_t code; int64_t idx; } or_kv;
static int or_kv_cmp(const void *pa, const void *pb)
{
    const or_kv *a = (const or_kv *)pa, *b = (const or_kv *)pb;
    if (a->code != b->code) return a->code < b->code ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Stable order by Morton code (ties by original index). */
void or_morton_sort(int n, const uint64_t *codes, int32_t *perm, uint64_t *sorted)
{
    or_kv *kv = (or_kv *)malloc(sizeof(or_kv) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) { kv[i].code = codes[i]; kv[i].idx = i; }
    qsort(kv, (size_t)n, sizeof(or_kv), or_kv_cmp);
    for (int i = 0; i < n; ++i) { perm[i] = (int32_t)kv[i].idx; sorted[i] = kv[i].code; }
    free(kv);
}

/* ------------------------------------------------------------------------ */
/* Cluster tree (Definition 1)                                               */
/* ------------------------------------------------------------------------ */

/* Nodes are numbered in breadth-first order.  A node is a leaf iff its size
 * is < leaf (Definition 1 (3), strict).  A node that is not a leaf is split
 * at the highest Morton bit on which its first and last codes differ (the
 * midpoint plane of its octree cell along that bit's axis); if all its codes
 * are equal it is split at begin + floor(size/2).  Boxes are the min/max of
 * the node's sorted centres.  Returns the node count (or -1 if cap is too
 * small). */
int or_build_tree(int n, const uint64_t *codes, const double *Xs, int leaf, int cap, int32_t *nbeg, int32_t *nend,
                  int32_t *child, int32_t *parent, double *lo, double *hi)
{
    if (n <= 0) return 0;
    int count = 1, head = 0;
    nbeg[0] = 0; nend[0] = n; parent[0] = -1;
    while (head < count) {
        int i = head++;
        int b = nbeg[i], e = nend[i], sz = e - b;
        child[2 * i] = child[2 * i + 1] = -1;
        if (sz >= leaf) {
            uint64_t d = codes[b] ^ codes[e - 1];
            int s;
            if (d == 0) {
                s = b + sz / 2;
            } else {
                int bit = 63;
                while (!((d >> bit) & 1u)) --bit;
                s = b;
                while (s < e && !((codes[s] >> bit) & 1u)) ++s;
            }
            if (count + 2 > cap) return -1;
            child[2 * i] = count; child[2 * i + 1] = count + 1;
            nbeg[count] = b; nend[count] = s; parent[count] = i;
            nbeg[count + 1] = s; nend[count + 1] = e; parent[count + 1] = i;
            count += 2;
        }
    }
    for (int i = 0; i < count; ++i)
        for (int a = 0; a < 3; ++a) {
            double l = Xs[3 * (size_t)nbeg[i] + a], h = l;
            for (int m = nbeg[i] + 1; m < nend[i]; ++m) {
                double v = Xs[3 * (size_t)m + a];
                if (v < l) l = v;
                if (v > h) h = v;
            }
            lo[3 * i + a] = l; hi[3 * i + a] = h;
        }
    return count;
}

/* ------------------------------------------------------------------------ */
/* Admissibility (Eq. 7) and BuildPartition (Algorithm 1)                    */
/* ------------------------------------------------------------------------ */

/* Bounding-box reading of Eq. 7, compared in squared form:
 *   diam^2(t) = sum_a (hi_a - lo_a)^2,
 *   dist^2    = sum_a max(0, lo_s - hi_t, lo_t - hi_s)^2,
 *   admissible iff dist^2 > 0 and max(diam^2(t), diam^2(s)) <= (eta*eta) * dist^2.
 * Blocks whose boxes touch or overlap (dist = 0) are never admissible; without
 * that, a one-particle cluster paired with itself (diam = dist = 0) would pass
 * and its self pair would enter the low-rank part. */
int or_admissible(const double *lo, const double *hi, int t, int s, double eta)
{
    double dt = 0.0, ds = 0.0, g = 0.0;
    for (int a = 0; a < 3; ++a) {
        double et = hi[3 * t + a] - lo[3 * t + a];
        double es = hi[3 * s + a] - lo[3 * s + a];
        double g1 = lo[3 * s + a] - hi[3 * t + a];
        double g2 = lo[3 * t + a] - hi[3 * s + a];
        double gap = 0.0;
        if (g1 > gap) gap = g1;
        if (g2 > gap) gap = g2;
        dt = dt + et * et;
        ds = ds + es * es;
        g = g + gap * gap;
    }
    double dm = dt > ds ? dt : ds;
    double eta2 = eta * eta;
    return g > 0.0 && dm <= eta2 * g;
}

typedef struct {
    const int32_t *nbeg, *nend, *child;
    const double *lo, *hi;
    int leaf;
    double eta;
    int32_t *G; int64_t nG, capG;
    int32_t *H; int64_t nH, capH;
    int overflow;
} or_part_state;

static void or_push(int32_t *L, int64_t *n, int64_t cap, int *ovf, int t, int s)
{
    if (*n >= cap) { *ovf = 1; return; }
    L[2 * *n] = t; L[2 * *n + 1] = s; ++*n;
}

static void or_build_partition(or_part_state *st, int t, int s)
{
    int szt = st->nend[t] - st->nbeg[t], szs = st->nend[s] - st->nbeg[s];
    if (or_admissible(st->lo, st->hi, t, s, st->eta)) {
        or_push(st->G, &st->nG, st->capG, &st->overflow, t, s);
    } else if (szt < st->leaf && szs < st->leaf) {
        or_push(st->H, &st->nH, st->capH, &st->overflow, t, s);
    } else if (szs < st->leaf) {
        or_build_partition(st, st->child[2 * t], s);
        or_build_partition(st, st->child[2 * t + 1], s);
    } else if (szt < st->leaf) {
        or_build_partition(st, t, st->child[2 * s]);
        or_build_partition(st, t, st->child[2 * s + 1]);
    } else {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v) or_build_partition(st, st->child[2 * t + u], st->child[2 * s + v]);
    }
}

static int or_pair_cmp(const void *pa, const void *pb)
{
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    return a[1] < b[1] ? -1 : (a[1] > b[1]);
}

/* Partition from (root, root).  Both lists are returned sorted by (target,
 * source).  Returns 0, or -1 if a capacity was exceeded (nG / nH then hold
 * the counts reached). */
int or_partition(int n_nodes, const int32_t *nbeg, const int32_t *nend, const int32_t *child, const double *lo,
                 const double *hi, int leaf, double eta, int32_t *G, int64_t capG, int64_t *nG, int32_t *H,
                 int64_t capH, int64_t *nH)
{
    or_part_state st = {nbeg, nend, child, lo, hi, leaf, eta, G, 0, capG, H, 0, capH, 0};
    if (n_nodes > 0) or_build_partition(&st, 0, 0);
    *nG = st.nG; *nH = st.nH;
    if (st.overflow) return -1;
    qsort(G, (size_t)st.nG, 2 * sizeof(int32_t), or_pair_cmp);
    qsort(H, (size_t)st.nH, 2 * sizeof(int32_t), or_pair_cmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Block ACA (Algorithm 2) with 3x3 elements                                 */
/* ------------------------------------------------------------------------ */

static double or_fro2(const double *A) { double s = 0; for (int e = 0; e < 9; ++e) s += A[e] * A[e]; return s; }

static double or_det3(const double *P)
{
    return P[0] * (P[4] * P[8] - P[5] * P[7]) - P[1] * (P[3] * P[8] - P[5] * P[6]) +
           P[2] * (P[3] * P[7] - P[4] * P[6]);
}

/* Inverse by adjugate / determinant.  Returns det. */
static double or_inv3(const double *P, double *Pi)
{
    double det = or_det3(P);
    Pi[0] = (P[4] * P[8] - P[5] * P[7]) / det;
    Pi[1] = (P[2] * P[7] - P[1] * P[8]) / det;
    Pi[2] = (P[1] * P[5] - P[2] * P[4]) / det;
    Pi[3] = (P[5] * P[6] - P[3] * P[8]) / det;
    Pi[4] = (P[0] * P[8] - P[2] * P[6]) / det;
    Pi[5] = (P[2] * P[3] - P[0] * P[5]) / det;
    Pi[6] = (P[3] * P[7] - P[4] * P[6]) / det;
    Pi[7] = (P[1] * P[6] - P[0] * P[7]) / det;
    Pi[8] = (P[0] * P[4] - P[1] * P[3]) / det;
    return det;
}

static void or_mm3(const double *A, const double *B, double *Cm) /* Cm = A B */
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Cm[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

/* Block-entry callback: G(m, n) for block-local indices. */
typedef void (*or_entry_fn)(void *ctx, int m, int n, double K[9]);

typedef struct {
    const or_kernel *k;
    const double *Xs;
    int t0, s0;
} or_geo_entry_ctx;

static void or_geo_entry(void *vctx, int m, int n, double K[9])
{
    or_geo_entry_ctx *c = (or_geo_entry_ctx *)vctx;
    const double *xt = c->Xs + 3 * (size_t)(c->t0 + m), *xs = c->Xs + 3 * (size_t)(c->s0 + n);
    double r[3] = {xt[0] - xs[0], xt[1] - xs[1], xt[2] - xs[2]};
    or_pair_block(c->k, r, K);
}

typedef struct { const double *G; int q; } or_dense_entry_ctx;
static void or_dense_entry(void *vctx, int m, int n, double K[9])
{
    or_dense_entry_ctx *c = (or_dense_entry_ctx *)vctx;
    memcpy(K, c->G + 9 * ((size_t)m * c->q + n), 9 * sizeof(double));
}

/* Algorithm 2 on a c x q block of 3x3 elements.
 *  C: [max_rank][c][9], Q: [max_rank][q][9] (element (p, m) holds c_p(m) /
 *  q_p(n) row-major).  I, J: pivots (J[0] = j1).  Returns the rank l.
 *  *flags |= 1 if the loop stopped at max_rank without meeting Eq. 10.
 *  lambda2 receives the running lambda^2 of Algorithm 2.
 * Readings: pivot measure = Frobenius norm (the algorithm's, not the
 * determinant the text of Eq. 9 mentions); ties go to the lowest local index;
 * the column is right-multiplied by the inverse of its pivot element; the
 * stop test nu^2 <= zeta^2 lambda^2 is applied after appending the pair;
 * if the selected pivot element is singular or badly conditioned
 * (1/(|P|_F |P^-1|_F) < 1e-10) the eligible row with the largest |det| is
 * used instead; a zero column residual, or no non-singular eligible pivot,
 * ends the loop with the pairs found so far. */
static int or_aca_core(or_entry_fn entry, void *ectx, int c, int q, double eps, int max_rank, int j1, double *C,
                       double *Q, int32_t *I, int32_t *J, double *lambda2, int *flags)
{
    char *usedR = (char *)calloc((size_t)c, 1), *usedC = (char *)calloc((size_t)q, 1);
    double *r = (double *)malloc(sizeof(double) * 9 * (size_t)c);
    double *A = (double *)malloc(sizeof(double) * 9 * (size_t)(max_rank > 0 ? max_rank : 1));
    double *B = (double *)malloc(sizeof(double) * 9 * (size_t)(max_rank > 0 ? max_rank : 1));
    int kmax = c < q ? c : q;
    if (kmax > max_rank) kmax = max_rank;
    double lam2 = 0.0;
    int k = 0, converged = 0, j = j1;
    usedC[j] = 1;
    while (k < kmax) {
        /* line 4: column residual c_k = G(:, j_k) - C Q(:, j_k) */
        for (int m = 0; m < c; ++m) {
            double g[9];
            entry(ectx, m, j, g);
            for (int p = 0; p < k; ++p) {
                double t[9];
                or_mm3(C + 9 * ((size_t)p * c + m), Q + 9 * ((size_t)p * q + j), t);
                for (int e = 0; e < 9; ++e) g[e] -= t[e];
            }
            memcpy(r + 9 * (size_t)m, g, sizeof g);
        }
        /* line 5: row pivot */
        int i = -1;
        double best = -1.0;
        for (int m = 0; m < c; ++m) {
            if (usedR[m]) continue;
            double v = or_fro2(r + 9 * (size_t)m);
            if (v > best) { best = v; i = m; }
        }
        if (i < 0 || !(best > 0.0)) { converged = 1; break; }
        double Pi[9];
        double det = or_inv3(r + 9 * (size_t)i, Pi);
        double rc = (det != 0.0) ? 1.0 / sqrt(or_fro2(r + 9 * (size_t)i) * or_fro2(Pi)) : 0.0;
        if (!(det != 0.0) || !(rc >= 1e-10)) {
            double bd = 0.0;
            int bi = -1;
            for (int m = 0; m < c; ++m) {
                if (usedR[m]) continue;
                double dv = fabs(or_det3(r + 9 * (size_t)m));
                if (dv > bd) { bd = dv; bi = m; }
            }
            if (bi < 0) { converged = 1; break; }
            i = bi;
            or_inv3(r + 9 * (size_t)i, Pi);
        }
        usedR[i] = 1;
        I[k] = i;
        J[k] = j;
        /* line 6: c_k = c_k [c_k(i_k)]^-1 */
        double *Ck = C + 9 * (size_t)k * c;
        for (int m = 0; m < c; ++m) or_mm3(r + 9 * (size_t)m, Pi, Ck + 9 * (size_t)m);
        /* line 7: row residual q_k = G(i_k, :) - C(i_k, :) Q */
        double *Qk = Q + 9 * (size_t)k * q;
        for (int n = 0; n < q; ++n) {
            double g[9];
            entry(ectx, i, n, g);
            for (int p = 0; p < k; ++p) {
                double t[9];
                or_mm3(C + 9 * ((size_t)p * c + i), Q + 9 * ((size_t)p * q + n), t);
                for (int e = 0; e < 9; ++e) g[e] -= t[e];
            }
            memcpy(Qk + 9 * (size_t)n, g, sizeof g);
        }
        /* line 8: next column pivot */
        int jn = -1;
        best = -1.0;
        for (int n = 0; n < q; ++n) {
            if (usedC[n]) continue;
            double v = or_fro2(Qk + 9 * (size_t)n);
            if (v > best) { best = v; jn = n; }
        }
        /* lines 9-10: nu^2 and lambda^2 with 3x3 Gram matrices
         *   A_pk = sum_m c_p(m)^T c_k(m),  B_kp = sum_n q_k(n) q_p(n)^T,
         *   nu^2 = tr(A_kk B_kk),  lambda^2 += nu^2 + 2 sum_{p<k} tr(A_pk B_kp). */
        for (int p = 0; p <= k; ++p) {
            double *Ap = A + 9 * p, *Bp = B + 9 * p;
            for (int e = 0; e < 9; ++e) { Ap[e] = 0.0; Bp[e] = 0.0; }
            for (int m = 0; m < c; ++m) {
                const double *cp = C + 9 * ((size_t)p * c + m), *ck = Ck + 9 * (size_t)m;
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y)
                        Ap[3 * x + y] += cp[x] * ck[y] + cp[3 + x] * ck[3 + y] + cp[6 + x] * ck[6 + y];
            }
            for (int nn = 0; nn < q; ++nn) {
                const double *qp = Q + 9 * ((size_t)p * q + nn), *qk = Qk + 9 * (size_t)nn;
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y)
                        Bp[3 * x + y] += qk[3 * x] * qp[3 * y] + qk[3 * x + 1] * qp[3 * y + 1] + qk[3 * x + 2] * qp[3 * y + 2];
            }
        }
        double nu2 = 0.0, cross = 0.0;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) nu2 += A[9 * k + 3 * x + y] * B[9 * k + 3 * y + x];
        for (int p = 0; p < k; ++p)
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) cross += A[9 * p + 3 * x + y] * B[9 * p + 3 * y + x];
        lam2 = lam2 + nu2 + 2.0 * cross;
        ++k;
        /* line 12 (Eq. 10, squared): stop when nu <= zeta lambda */
        if (nu2 <= eps * eps * lam2) { converged = 1; break; }
        if (jn < 0) { converged = 1; break; }
        usedC[jn] = 1;
        j = jn;
    }
    if (!converged && k == max_rank && k < (c < q ? c : q)) *flags |= 1;
    *lambda2 = lam2;
    free(usedR); free(usedC); free(r); free(A); free(B);
    return k;
}

/* ACA of the geometric block (targets Xs[t0 .. t0+c), sources Xs[s0 .. s0+q)). */
int or_aca_block(const or_kernel *k, const double *Xs, int t0, int c, int s0, int q, double eps, int max_rank, int j1,
                 double *C, double *Q, int32_t *I, int32_t *J, double *lambda2, int *flags)
{
    or_geo_entry_ctx ctx = {k, Xs, t0, s0};
    return or_aca_core(or_geo_entry, &ctx, c, q, eps, max_rank, j1, C, Q, I, J, lambda2, flags);
}

/* ACA of an explicit block G [c][q][9] (for checks against the SVD). */
int or_aca_dense(const double *G, int c, int q, double eps, int max_rank, int j1, double *C, double *Q, int32_t *I,
                 int32_t *J, double *lambda2, int *flags)
{
    or_dense_entry_ctx ctx = {G, q};
    return or_aca_core(or_dense_entry, &ctx, c, q, eps, max_rank, j1, C, Q, I, J, lambda2, flags);
}

/* ------------------------------------------------------------------------ */
/* Short-range terms: M^(s,2), M^(t,3), M^(s,3) of Eq. 6                    */
/* ------------------------------------------------------------------------ */

/* MLP n_in -> w -> w -> w -> n_out, SiLU after each hidden layer, linear
 * output; parameters packed per layer as W [out, in] then b [out]. */
void or_mlp_gen(const double *theta, int n_in, int w, int n_out, const double *f, double *o)
{
    double h[256], g[256];
    const double *p = theta;
    p = or_layer(p, n_in, w, f, h);
    for (int i = 0; i < w; ++i) h[i] = or_silu(h[i]);
    p = or_layer(p, w, w, h, g);
    for (int i = 0; i < w; ++i) g[i] = or_silu(g[i]);
    p = or_layer(p, w, w, g, h);
    for (int i = 0; i < w; ++i) h[i] = or_silu(h[i]);
    or_layer(p, w, n_out, h, o);
}

/* Neighbour lists N(i) = { j != i : |x_i - x_j| < rcut } by brute force
 * (CSR: off[n+1], idx in increasing j). */
static void or_neighbours(int n, const double *X, double rcut, int64_t **off_out, int32_t **idx_out)
{
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    const double rc2 = rcut * rcut;
    for (int i = 0; i < n; ++i) {
        int64_t cnt = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = X[3 * i] - X[3 * j], dy = X[3 * i + 1] - X[3 * j + 1], dz = X[3 * i + 2] - X[3 * j + 2];
            if (dx * dx + dy * dy + dz * dz < rc2) ++cnt;
        }
        off[i + 1] = off[i] + cnt;
    }
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[n] > 0 ? off[n] : 1));
    for (int i = 0; i < n; ++i) {
        int64_t w = off[i];
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = X[3 * i] - X[3 * j], dy = X[3 * i + 1] - X[3 * j + 1], dz = X[3 * i + 2] - X[3 * j + 2];
            if (dx * dx + dy * dy + dz * dz < rc2) idx[w++] = j;
        }
    }
    *off_out = off;
    *idx_out = idx;
}

/* U_i += sum over the short-range terms of Eq. 2 (Eq. 6: M^(s,2) + M^(t,3)
 * + M^(s,3)) with the normalisations of Eq. 4, for one suspension of n
 * particles (added to U, FP64):
 *   two-body self part, j in N(i), r = x_i - x_j, d = |r|:
 *     alpha2s = (a/d)^4 / d * S(MLP_s([r/d, a/d]))   applied to F_i;
 *   three-body, 3-cliques (j, k, i) with i, j in N(k), j != i (k in N(i),
 *   j in N(k) \ {i}), r_ji = x_j - x_i, r_ki = x_k - x_i, d_jk = |x_j - x_k|:
 *     o = MLP_3([r_ji/|r_ji|, r_ki/|r_ki|, a/d_jk]) (12 outputs),
 *     alpha3 = [S(o_0..5), S(o_6..11)] / (d_jk |r_ki|)  applied to [F_i; F_j].
 * theta_s: MLP 4 -> ws -> ws -> ws -> 6; theta_3: MLP 7 -> w3 -> w3 -> w3 -> 12
 * (either may be NULL to leave its term out). */
void or_short_range(int n, const double *X, const double *F, const double *theta_s, int ws, const double *theta_3,
                    int w3, double rcut, double a, double *U)
{
    int64_t *off;
    int32_t *idx;
    or_neighbours(n, X, rcut, &off, &idx);
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        double ui[3] = {0.0, 0.0, 0.0};
        const double *xi = X + 3 * i, *Fi = F + 3 * i;
        if (theta_s) {
            for (int64_t e = off[i]; e < off[i + 1]; ++e) {
                const int j = idx[e];
                double r[3] = {xi[0] - X[3 * j], xi[1] - X[3 * j + 1], xi[2] - X[3 * j + 2]};
                double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                double f[4] = {r[0] / d, r[1] / d, r[2] / d, a / d};
                double o[6], S[9];
                or_mlp_gen(theta_s, 4, ws, 6, f, o);
                or_sym3(o, S);
                double q = a / d, c = q * q * q * q / d;
                for (int u = 0; u < 3; ++u) ui[u] += c * (S[3 * u] * Fi[0] + S[3 * u + 1] * Fi[1] + S[3 * u + 2] * Fi[2]);
            }
        }
        if (theta_3) {
            for (int64_t e = off[i]; e < off[i + 1]; ++e) {
                const int k = idx[e];
                double rki[3] = {X[3 * k] - xi[0], X[3 * k + 1] - xi[1], X[3 * k + 2] - xi[2]};
                double dki = sqrt(rki[0] * rki[0] + rki[1] * rki[1] + rki[2] * rki[2]);
                for (int64_t e2 = off[k]; e2 < off[k + 1]; ++e2) {
                    const int j = idx[e2];
                    if (j == i) continue;
                    double rji[3] = {X[3 * j] - xi[0], X[3 * j + 1] - xi[1], X[3 * j + 2] - xi[2]};
                    double dji = sqrt(rji[0] * rji[0] + rji[1] * rji[1] + rji[2] * rji[2]);
                    double djk[3] = {X[3 * j] - X[3 * k], X[3 * j + 1] - X[3 * k + 1], X[3 * j + 2] - X[3 * k + 2]};
                    double dj = sqrt(djk[0] * djk[0] + djk[1] * djk[1] + djk[2] * djk[2]);
                    double f[7] = {rji[0] / dji, rji[1] / dji, rji[2] / dji, rki[0] / dki, rki[1] / dki, rki[2] / dki,
                                   a / dj};
                    double o[12], Ss[9], St[9];
                    or_mlp_gen(theta_3, 7, w3, 12, f, o);
                    or_sym3(o, Ss);
                    or_sym3(o + 6, St);
                    const double *Fj = F + 3 * j;
                    double c = 1.0 / (dj * dki);
                    for (int u = 0; u < 3; ++u)
                        ui[u] += c * (Ss[3 * u] * Fi[0] + Ss[3 * u + 1] * Fi[1] + Ss[3 * u + 2] * Fi[2] +
                                      St[3 * u] * Fj[0] + St[3 * u + 1] * Fj[1] + St[3 * u + 2] * Fj[2]);
                }
            }
        }
        for (int u = 0; u < 3; ++u) U[3 * i + u] += ui[u];
    }
    free(off);
    free(idx);
}

/* ------------------------------------------------------------------------ */
/* H-matrix product                                                          */
/* ------------------------------------------------------------------------ */

/* j1 for a block (the paper draws it at random): rule 0 = first source
 * (local index 0); rule 1 = splitmix64(seed ^ (t << 32) ^ s) mod q. */
static uint64_t or_splitmix_once(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int or_j1(int rule, uint64_t seed, int t, int s, int q)
{
    if (rule == 0 || q <= 1) return 0;
    uint64_t h = or_splitmix_once(seed ^ ((uint64_t)(uint32_t)t << 32) ^ (uint64_t)(uint32_t)s);
    return (int)(h % (uint64_t)q);
}

typedef struct {
    int64_t n_nodes, nG, nH;
    int64_t n_near_pairs, n_aca_entries, rank_sum, rank_max, rank_capped;
} or_hstats;

/* U = alpha_1 F + M_H F where M_H is the H-matrix of M^(t,2): tree, partition,
 * dense inadmissible blocks (self pair skipped) and ACA on admissible blocks,
 * each applied as C (Q F_sigma) (Section 3, Eq. 8).  X, F, U in the caller's
 * order.  ranks (optional, length >= nG) receives each admissible block's
 * rank in the sorted block order; pivI/pivJ (optional, nG*max_rank) receive
 * the pivots.  Returns 0 or a negative error. */
int or_hmatvec(int n, const double *X, const double *F, const or_kernel *k, int leaf, double eta, double eps,
               int max_rank, int j1_rule, uint64_t seed, int with_self, double *U, or_hstats *stats, int32_t *ranks,
               int32_t *pivI, int32_t *pivJ, int64_t ranks_cap)
{
    if (n <= 0) return 0;
    uint64_t *codes = (uint64_t *)malloc(8 * (size_t)n), *sc = (uint64_t *)malloc(8 * (size_t)n);
    int32_t *perm = (int32_t *)malloc(4 * (size_t)n);
    or_morton_codes(n, X, codes);
    or_morton_sort(n, codes, perm, sc);
    double *Xs = (double *)malloc(24 * (size_t)n), *Fs = (double *)malloc(24 * (size_t)n);
    for (int m = 0; m < n; ++m)
        for (int a = 0; a < 3; ++a) { Xs[3 * m + a] = X[3 * perm[m] + a]; Fs[3 * m + a] = F[3 * perm[m] + a]; }
    int cap = 2 * n + 1;
    int32_t *nb = (int32_t *)malloc(4 * (size_t)cap), *ne = (int32_t *)malloc(4 * (size_t)cap);
    int32_t *ch = (int32_t *)malloc(8 * (size_t)cap), *par = (int32_t *)malloc(4 * (size_t)cap);
    double *lo = (double *)malloc(24 * (size_t)cap), *hi = (double *)malloc(24 * (size_t)cap);
    int nn = or_build_tree(n, sc, Xs, leaf, cap, nb, ne, ch, par, lo, hi);
    int64_t capG = 1 << 16, capH = 1 << 16, nG = 0, nH = 0;
    int32_t *G = NULL, *H = NULL;
    for (;;) {
        G = (int32_t *)malloc(8 * (size_t)capG);
        H = (int32_t *)malloc(8 * (size_t)capH);
        if (or_partition(nn, nb, ne, ch, lo, hi, leaf, eta, G, capG, &nG, H, capH, &nH) == 0) break;
        free(G); free(H);
        capG *= 4; capH *= 4;
    }
    double *y = (double *)calloc(3 * (size_t)n, sizeof(double));
    int64_t near_pairs = 0, aca_entries = 0, rank_sum = 0, rank_max = 0, capped = 0;
    /* inadmissible blocks: dense, self pair excluded; blocks sharing a target
     * are contiguous (sorted), so rows are parallel over targets. */
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : near_pairs)
    for (int64_t b = 0; b < nH; ++b) {
        if (b > 0 && H[2 * b] == H[2 * (b - 1)]) continue;
        int t = H[2 * b];
        for (int64_t bb = b; bb < nH && H[2 * bb] == t; ++bb) {
            int s = H[2 * bb + 1];
            for (int m = nb[t]; m < ne[t]; ++m)
                for (int j = nb[s]; j < ne[s]; ++j) {
                    if (m == j) continue;
                    double r[3] = {Xs[3 * m] - Xs[3 * j], Xs[3 * m + 1] - Xs[3 * j + 1], Xs[3 * m + 2] - Xs[3 * j + 2]};
                    double K[9];
                    or_pair_block(k, r, K);
                    for (int a = 0; a < 3; ++a)
                        y[3 * m + a] += K[3 * a] * Fs[3 * j] + K[3 * a + 1] * Fs[3 * j + 1] + K[3 * a + 2] * Fs[3 * j + 2];
                    ++near_pairs;
                }
        }
    }
    /* admissible blocks: ACA then C (Q F) into a per-block partial */
    int64_t *pofs = (int64_t *)malloc(8 * (size_t)(nG + 1));
    pofs[0] = 0;
    for (int64_t b = 0; b < nG; ++b) pofs[b + 1] = pofs[b] + 3 * (int64_t)(ne[G[2 * b]] - nb[G[2 * b]]);
    double *part = (double *)calloc((size_t)pofs[nG] + 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : aca_entries, rank_sum, capped) reduction(max : rank_max)
    for (int64_t b = 0; b < nG; ++b) {
        int t = G[2 * b], s = G[2 * b + 1];
        int c = ne[t] - nb[t], q = ne[s] - nb[s];
        double *Cf = (double *)malloc(sizeof(double) * 9 * (size_t)c * max_rank);
        double *Qf = (double *)malloc(sizeof(double) * 9 * (size_t)q * max_rank);
        int32_t *Ib = (int32_t *)malloc(4 * (size_t)max_rank), *Jb = (int32_t *)malloc(4 * (size_t)max_rank);
        double l2;
        int fl = 0;
        int j1 = or_j1(j1_rule, seed, t, s, q);
        int l = or_aca_block(k, Xs, nb[t], c, nb[s], q, eps, max_rank, j1, Cf, Qf, Ib, Jb, &l2, &fl);
        if (ranks && b < ranks_cap) ranks[b] = l;
        if (pivI && b < ranks_cap)
            for (int p = 0; p < max_rank; ++p) {
                pivI[b * max_rank + p] = p < l ? Ib[p] : -1;
                pivJ[b * max_rank + p] = p < l ? Jb[p] : -1;
            }
        aca_entries += (int64_t)(c + q) * l;
        rank_sum += l;
        if (l > rank_max) rank_max = l;
        capped += fl & 1;
        double *tv = (double *)malloc(sizeof(double) * 3 * (size_t)(l > 0 ? l : 1));
        for (int p = 0; p < l; ++p) {
            double acc[3] = {0, 0, 0};
            for (int jj = 0; jj < q; ++jj) {
                const double *Qe = Qf + 9 * ((size_t)p * q + jj), *fj = Fs + 3 * (size_t)(nb[s] + jj);
                for (int a = 0; a < 3; ++a) acc[a] += Qe[3 * a] * fj[0] + Qe[3 * a + 1] * fj[1] + Qe[3 * a + 2] * fj[2];
            }
            for (int a = 0; a < 3; ++a) tv[3 * p + a] = acc[a];
        }
        double *pb = part + pofs[b];
        for (int m = 0; m < c; ++m) {
            double acc[3] = {0, 0, 0};
            for (int p = 0; p < l; ++p) {
                const double *Ce = Cf + 9 * ((size_t)p * c + m), *tp = tv + 3 * p;
                for (int a = 0; a < 3; ++a) acc[a] += Ce[3 * a] * tp[0] + Ce[3 * a + 1] * tp[1] + Ce[3 * a + 2] * tp[2];
            }
            for (int a = 0; a < 3; ++a) pb[3 * m + a] = acc[a];
        }
        free(tv); free(Cf); free(Qf); free(Ib); free(Jb);
    }
    for (int64_t b = 0; b < nG; ++b) {
        int t = G[2 * b];
        for (int m = 0; m < ne[t] - nb[t]; ++m)
            for (int a = 0; a < 3; ++a) y[3 * (size_t)(nb[t] + m) + a] += part[pofs[b] + 3 * m + a];
    }
    double a1 = or_self_mobility(k->a, k->mu);
    for (int m = 0; m < n; ++m)
        for (int a = 0; a < 3; ++a) U[3 * (size_t)perm[m] + a] = (with_self ? a1 * Fs[3 * m + a] : 0.0) + y[3 * m + a];
    if (stats) {
        stats->n_nodes = nn; stats->nG = nG; stats->nH = nH;
        stats->n_near_pairs = near_pairs; stats->n_aca_entries = aca_entries;
        stats->rank_sum = rank_sum; stats->rank_max = rank_max; stats->rank_capped = capped;
    }
    free(codes); free(sc); free(perm); free(Xs); free(Fs); free(nb); free(ne); free(ch); free(par);
    free(lo); free(hi); free(G); free(H); free(y); free(pofs); free(part);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Filament suspension: bead forces (Section 4.3, filament application)    */
/* ------------------------------------------------------------------------ */

/* Chains of `beads` consecutive rows of X.  Energy (reading: the paper's bond
 * spring of Eq. 12 and a bending term whose printed force is garbled, taken
 * from the stated potential):
 *   E = sum_bonds (k/2)(|r| - l0)^2 + sum_joints kappa (1 - t_a . t_b)
 *       - sum_beads g . x
 * with r = x_{j+1} - x_j along each chain and t = r / |r|. */
double or_filament_energy(int n_chains, int beads, const double *X, double k, double l0, double kappa,
                          const double *g)
{
    double e = 0.0;
    for (int c = 0; c < n_chains; ++c) {
        const double *x = X + (int64_t)3 * c * beads;
        for (int j = 0; j + 1 < beads; ++j) {
            double r[3], L = 0.0;
            for (int d = 0; d < 3; ++d) { r[d] = x[3 * (j + 1) + d] - x[3 * j + d]; L += r[d] * r[d]; }
            L = sqrt(L);
            e += 0.5 * k * (L - l0) * (L - l0);
        }
        for (int j = 0; j + 2 < beads; ++j) {
            double ra[3], rb[3], La = 0.0, Lb = 0.0, dot = 0.0;
            for (int d = 0; d < 3; ++d) {
                ra[d] = x[3 * (j + 1) + d] - x[3 * j + d];
                rb[d] = x[3 * (j + 2) + d] - x[3 * (j + 1) + d];
                La += ra[d] * ra[d];
                Lb += rb[d] * rb[d];
            }
            La = sqrt(La);
            Lb = sqrt(Lb);
            for (int d = 0; d < 3; ++d) dot += (ra[d] / La) * (rb[d] / Lb);
            e += kappa * (1.0 - dot);
        }
    }
    for (int64_t i = 0; i < (int64_t)n_chains * beads; ++i)
        for (int d = 0; d < 3; ++d) e -= g[d] * X[3 * i + d];
    return e;
}

/* F = -grad E, accumulated term by term: each bond and each joint adds its
 * equal and opposite contributions to the beads it joins.
 *   bond:  dE/dr = k (|r| - l0) t
 *   joint: dE/dr_a = -kappa (t_b - (t_a.t_b) t_a) / |r_a|,
 *          dE/dr_b = -kappa (t_a - (t_a.t_b) t_b) / |r_b|
 * and a bond r = x_{j+1} - x_j passes dE/dr to x_{j+1} and -dE/dr to x_j. */
void or_filament_forces(int n_chains, int beads, const double *X, double k, double l0, double kappa,
                        const double *g, double *F)
{
    for (int64_t i = 0; i < (int64_t)n_chains * beads; ++i)
        for (int d = 0; d < 3; ++d) F[3 * i + d] = g[d];
    for (int c = 0; c < n_chains; ++c) {
        const double *x = X + (int64_t)3 * c * beads;
        double *f = F + (int64_t)3 * c * beads;
        for (int j = 0; j + 1 < beads; ++j) {
            double r[3], L = 0.0;
            for (int d = 0; d < 3; ++d) { r[d] = x[3 * (j + 1) + d] - x[3 * j + d]; L += r[d] * r[d]; }
            L = sqrt(L);
            for (int d = 0; d < 3; ++d) {
                double dEdr = k * (L - l0) * (r[d] / L);
                f[3 * (j + 1) + d] -= dEdr;
                f[3 * j + d] += dEdr;
            }
        }
        for (int j = 0; j + 2 < beads; ++j) {
            double ta[3], tb[3], La = 0.0, Lb = 0.0, cs = 0.0;
            for (int d = 0; d < 3; ++d) {
                ta[d] = x[3 * (j + 1) + d] - x[3 * j + d];
                tb[d] = x[3 * (j + 2) + d] - x[3 * (j + 1) + d];
                La += ta[d] * ta[d];
                Lb += tb[d] * tb[d];
            }
            La = sqrt(La);
            Lb = sqrt(Lb);
            for (int d = 0; d < 3; ++d) { ta[d] /= La; tb[d] /= Lb; }
            for (int d = 0; d < 3; ++d) cs += ta[d] * tb[d];
            for (int d = 0; d < 3; ++d) {
                double dEa = -kappa * (tb[d] - cs * ta[d]) / La;   /* bond a: x_j -> x_{j+1}     */
                double dEb = -kappa * (ta[d] - cs * tb[d]) / Lb;   /* bond b: x_{j+1} -> x_{j+2} */
                f[3 * (j + 1) + d] -= dEa;
                f[3 * j + d] += dEa;
                f[3 * (j + 2) + d] -= dEb;
                f[3 * (j + 1) + d] += dEb;
            }
        }
    }
}

/* Eq. 11: || a - b ||_2 / || a ||_2 over all components. */
double or_rel_error(int64_t n3, const double *ref, const double *approx)
{
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n3; ++i) {
        double d = ref[i] - approx[i];
        num += d * d;
        den += ref[i] * ref[i];
    }
    return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
