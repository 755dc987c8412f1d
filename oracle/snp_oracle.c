/*
 * snp_oracle.c -- FP64 CPU oracle for the splattable-neural-primitive tile
 * rasterizer (arXiv 2510.08491, "Splat the Net").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code, header,
 * table or constant generator with the CUDA path; the two meet only through the
 * seeded inputs of paper_2510_08491_gb300/synth.py.
 *
 * Plain, slow and written to be checked against the paper by eye:
 *   - Sec. 3.1, Eq. 5/6: density sigma(x) = W2 cos(w0 (W1 u + b1)) + b2 with
 *     u = (x - c)/||s||_inf (centred, isotropically scaled, not rotated).
 *   - Sec. 3.2: analytic ray/ellipsoid entry and exit t_in, t_out.
 *   - Sec. 3.2, Eq. 7/8: alpha_hat = S(t_out) - S(t_in) with the closed-form
 *     antiderivative S, the Eq. 5 normalisation folded into W1 and b1.
 *     Two algebraically equal forms: "naive" (Eq. 8 literally, a difference of
 *     sines divided by w0 W1 d / m) and "stable" (sin A - sin B =
 *     2 cos((A+B)/2) sin((A-B)/2), i.e. Delta_t * [b2 + sum w2 cos(phi_mid) sinc(theta)]).
 *   - Sec. 3.2, Eq. 9: alpha = 1 - exp(-max(0, alpha_hat)).
 *   - Sec. 2.1, Eq. 4: front-to-back alpha blending over depth-sorted primitives.
 *   - App. D.2 (Eq. color_render): per-primitive colour MLP, here with input
 *     [view direction, 8-d feature], two hidden ReLU layers, sigmoid output.
 *   - Sec. 3.1 / 3.3 (Primitives): view-dependent colour in four bands of real
 *     spherical harmonics (48 coefficients), evaluated along the direction from
 *     the camera to the primitive centre: c = max(0, 1/2 + sum_i Y_i(d) k_i).
 *   - App. Applications (volumetric dynamic scenes): time-conditioned density,
 *     the cosine argument gains xi_t W_t; the degree-0 SH coefficient follows a
 *     polynomial plus Fourier series in xi_t.
 *
 * Readings where the paper is silent (camera model, depth key, near plane, early
 * termination, tile keys) are the library's documented conventions; each one is
 * restated at its point of use below.
 *
 * The FP32 "key specification" (key_* functions) defines which primitives are
 * visible, their pixel rectangle and their depth key.  It is evaluated in IEEE
 * binary32 with every operation written out in a fixed order (+, -, *, /, sqrt
 * only; compiled with -ffp-contract=off), so an independent implementation that
 * follows the same written order produces bit-identical tile keys.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_COLOR_CONST 0
#define ORA_COLOR_MLP 1
#define ORA_COLOR_SH 2
#define ORA_FORM_STABLE 0
#define ORA_FORM_NAIVE 1
#define ORA_FEAT 8

/* Scene for the FP64 renderer: every array in float64 (the float32 inputs
 * converted exactly, or exactly perturbed values for finite differences). */
typedef struct {
    int64_t n;
    int32_t n_sigma;
    int32_t color_mode;
    int32_t n_c;
    int32_t pad_;
    double omega0;
    const double *centers, *log_scales, *quats; /* [n,3] [n,3] [n,4] (w,x,y,z) */
    const double *W1, *b1, *w2, *b2;            /* [n,Ns,3] [n,Ns] [n,Ns] [n] */
    const double *rgb;                          /* [n,3] */
    const double *feat, *Wc1, *bc1, *Wc2, *bc2, *Wc3, *bc3; /* [n,8] [n,Nc,11] [n,Nc] [n,Nc,Nc] [n,Nc] [n,3,Nc] [n,3] */
    const double *sh;                           /* [n,16,3] spherical-harmonic coefficients */
    /* Time-conditioned scenes (App. Applications, volumetric dynamic scenes); NULL
     * for static ones.  time = xi_t of the view being rendered (ora_render takes it
     * from the camera). */
    double time;
    const double *wt;                           /* [n,Ns] phase weights W_t */
    const double *sh_t;                         /* [n,12,3] degree-0 series a_1..4, b_1..4, c_1..4 */
} ora_scene;

/* Geometry for the FP32 key specification (the float32 inputs as given). */
typedef struct {
    int64_t n;
    const float *centers, *log_scales, *quats;
} ora_geom32;

typedef struct {
    float R_wc[9]; /* world -> camera, row-major; rows = camera x (right), y (down), z (forward) */
    float eye[3];
    float fx, fy, cx, cy, z_near;
    int32_t width, height;
    float time; /* xi_t of this view (dynamic scenes) */
} ora_camera;

/* =========================================================================
 * FP32 key specification (bit-exact part).
 * ========================================================================= */

/* exp in binary32 by Cody-Waite range reduction x = n ln2 + r (ln2 split into a
 * 16-bit head and a tail so that n * head is exact) and the degree-7 Taylor
 * polynomial of e^r in Horner form, then an exact scaling by 2^n.  Used for the
 * ellipsoid scales s = exp(log_s) on the key path so that both implementations
 * round identically. */
static float key_exp(float x)
{
    if (x > 80.0f) x = 80.0f;
    if (x < -80.0f) x = -80.0f;
    const float log2e = 0x1.715476p+0f;
    const float ln2_hi = 0x1.62e4p-1f;
    const float ln2_lo = 0x1.7f7d1cp-20f;
    float n = rintf(x * log2e);
    float r = x - n * ln2_hi;
    r = r - n * ln2_lo;
    float p = 0x1.a01a02p-13f;          /* 1/7! */
    p = 0x1.6c16c2p-10f + r * p;        /* 1/6! */
    p = 0x1.111112p-7f + r * p;         /* 1/5! */
    p = 0x1.555556p-5f + r * p;         /* 1/4! */
    p = 0x1.555556p-3f + r * p;         /* 1/3! */
    p = 0.5f + r * p;
    p = 1.0f + r * p;
    p = 1.0f + r * p;
    int32_t e = (int32_t)n + 127;
    uint32_t bits = (uint32_t)e << 23;
    float scale;
    memcpy(&scale, &bits, 4);
    return p * scale;
}

typedef struct {
    int32_t visible;
    int32_t px0, py0, px1, py1; /* inclusive pixel-index rectangle (pixel centres) */
    float depth;                /* camera-frame z of the centre */
} ora_keyrec;

/* Half-open pixel range of one image axis covered by the silhouette of the
 * ellipsoid {mu + V v : |v| <= 1} (camera frame, Sigma = V V^T).  The tangent
 * plane through the eye containing image column U has normal n = (f, 0, cc - U);
 * tangency is (n . mu)^2 = n^T Sigma n, a quadratic in p = cc - U:
 *   p^2 (mz^2 - Szz) + 2 p f (ma mz - Saz) + f^2 (ma^2 - Saa) = 0,
 * whose discriminant / 4 is f^2 (mz^2 Saa + ma^2 Szz - 2 ma mz Saz + Saz^2 - Saa Szz). */
#define KEY_EPS 0.03125f
static int key_bound(float f, float cc, float ma, float mz, float saa, float saz, float szz,
                     int32_t npx, int32_t *lo, int32_t *hi)
{
    float mzz = mz * mz;
    float a = mzz - szz;
    float maz = ma * mz;
    float bq = f * (maz - saz);
    float t1 = mzz * saa;
    float maa = ma * ma;
    float t2 = maa * szz;
    float t3 = 2.0f * (maz * saz);
    float t4 = saz * saz;
    float t5 = saa * szz;
    float D = t1 + t2;
    D = D - t3;
    D = D + t4;
    D = D - t5;
    if (!(D > 0.0f)) D = 0.0f;
    float sq = f * sqrtf(D);
    float pmax = (sq - bq) / a;
    float pmin = (-bq - sq) / a;
    float umin = cc - pmax;
    float umax = cc - pmin;
    float fl = ceilf((umin - 0.5f) - KEY_EPS);
    float fh = floorf((umax - 0.5f) + KEY_EPS);
    float lim = (float)(npx - 1);
    if (fl < 0.0f) fl = 0.0f;
    if (fh > lim) fh = lim;
    if (!(fl <= fh)) return 0;
    *lo = (int32_t)fl;
    *hi = (int32_t)fh;
    return 1;
}

static void key_project(const ora_geom32 *S, const ora_camera *cam, int64_t i, ora_keyrec *out)
{
    const float *c = S->centers + 3 * i, *ls = S->log_scales + 3 * i, *q = S->quats + 4 * i;
    const float *W = cam->R_wc;
    float s[3] = {key_exp(ls[0]), key_exp(ls[1]), key_exp(ls[2])};
    float qq = q[0] * q[0];
    qq = qq + q[1] * q[1];
    qq = qq + q[2] * q[2];
    qq = qq + q[3] * q[3];
    float inv = 1.0f / sqrtf(qq);
    float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
    float V[3][3];
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) {
            float t = W[3 * a + 0] * R[0][j];
            t = t + W[3 * a + 1] * R[1][j];
            t = t + W[3 * a + 2] * R[2][j];
            V[a][j] = t * s[j];
        }
#define SIG(a, b) ((V[a][0] * V[b][0] + V[a][1] * V[b][1]) + V[a][2] * V[b][2])
    float sxx = SIG(0, 0), sxz = SIG(0, 2), szz = SIG(2, 2), syy = SIG(1, 1), syz = SIG(1, 2);
#undef SIG
    float dl[3] = {c[0] - cam->eye[0], c[1] - cam->eye[1], c[2] - cam->eye[2]};
    float mu[3];
    for (int a = 0; a < 3; ++a) {
        float t = W[3 * a + 0] * dl[0];
        t = t + W[3 * a + 1] * dl[1];
        t = t + W[3 * a + 2] * dl[2];
        mu[a] = t;
    }
    float m = s[0] > s[1] ? s[0] : s[1];
    m = m > s[2] ? m : s[2];
    out->depth = mu[2];
    out->visible = 0;
    out->px0 = out->py0 = 0;
    out->px1 = out->py1 = -1;
    /* near plane: the whole bounding ellipsoid lies beyond z_near */
    if (!((mu[2] - m) > cam->z_near)) return;
    int32_t x0, x1, y0, y1;
    if (!key_bound(cam->fx, cam->cx, mu[0], mu[2], sxx, sxz, szz, cam->width, &x0, &x1)) return;
    if (!key_bound(cam->fy, cam->cy, mu[1], mu[2], syy, syz, szz, cam->height, &y0, &y1)) return;
    out->visible = 1;
    out->px0 = x0;
    out->px1 = x1;
    out->py0 = y0;
    out->py1 = y1;
}

/* Key record of every primitive for one camera. */
void ora_key_project(const ora_geom32 *S, const ora_camera *cam, int32_t *visible, int32_t *rect4,
                     float *depth)
{
    int64_t n = S->n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        ora_keyrec r;
        key_project(S, cam, i, &r);
        visible[i] = r.visible;
        rect4[4 * i + 0] = r.px0;
        rect4[4 * i + 1] = r.py0;
        rect4[4 * i + 2] = r.px1;
        rect4[4 * i + 3] = r.py1;
        depth[i] = r.depth;
    }
}

/* The key-path exponential, exposed for its accuracy test. */
float ora_key_exp(float x) { return key_exp(x); }

/* =========================================================================
 * FP64 geometry, integral, colour and compositing.
 * ========================================================================= */

typedef struct {
    double Minv[3][3]; /* world offset -> unit-sphere coordinates: diag(1/s) R_q^T */
    double c[3];
    double m, inv_m;   /* ||s||_inf */
} prim64;

static void prim_setup(const ora_scene *S, int64_t i, prim64 *P)
{
    const double *c = S->centers + 3 * i, *ls = S->log_scales + 3 * i, *q = S->quats + 4 * i;
    double s[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
    double R[3][3] = {
        {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
        {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
        {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)},
    };
    /* ellipsoid = { c + R diag(s) v : |v| <= 1 }  =>  v = diag(1/s) R^T (x - c) */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P->Minv[a][b] = R[b][a] / s[a];
    for (int k = 0; k < 3; ++k) P->c[k] = c[k];
    P->m = fmax(fmax(s[0], s[1]), s[2]);
    P->inv_m = 1.0 / P->m;
}

/* Ray o + t d against the ellipsoid: |Minv (o + t d - c)|^2 = 1.  Returns 1 on a
 * hit with the midpoint tm and half chord length `half` (t_in = tm - half,
 * t_out = tm + half).  The closest-approach form p = o' + tm d', h^2 = 1 - |p|^2
 * is used instead of the raw discriminant. */
static int intersect(const prim64 *P, const double o[3], const double d[3], double *tm, double *half)
{
    double oc[3] = {o[0] - P->c[0], o[1] - P->c[1], o[2] - P->c[2]};
    double op[3], dp[3];
    for (int a = 0; a < 3; ++a) {
        op[a] = P->Minv[a][0] * oc[0] + P->Minv[a][1] * oc[1] + P->Minv[a][2] * oc[2];
        dp[a] = P->Minv[a][0] * d[0] + P->Minv[a][1] * d[1] + P->Minv[a][2] * d[2];
    }
    double A = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
    double B = op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2];
    double t = -B / A;
    double p[3] = {op[0] + t * dp[0], op[1] + t * dp[1], op[2] + t * dp[2]};
    double h2 = 1.0 - (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    *tm = t;
    if (!(h2 > 0.0)) {
        *half = 0.0;
        return 0;
    }
    *half = sqrt(h2 / A);
    return 1;
}

static double sinc(double x)
{
    if (fabs(x) < 1e-4) return 1.0 - x * x / 6.0;
    return sin(x) / x;
}

/* Phase offset of hidden unit k that is constant along every ray: xi_t W_t,k for a
 * time-conditioned scene (App. Applications: the density's cosine argument gains
 * xi_t W_t outside the w0 factor), else 0. */
static double time_phase(const ora_scene *S, int64_t i, int k)
{
    return S->wt ? S->time * S->wt[(size_t)i * S->n_sigma + k] : 0.0;
}

/* Integral of sigma along o + t d over [tm - half, tm + half], stable form:
 * phi_k = w0 (W1_k . u_mid + b1_k) (+ xi_t W_t,k), theta_k = w0 (W1_k . d) half / m,
 * alpha_hat = 2 half [b2 + sum_k w2_k cos(phi_k) sinc(theta_k)]. */
static double integral_stable(const ora_scene *S, int64_t i, const prim64 *P, const double o[3],
                              const double d[3], double tm, double half)
{
    int Ns = S->n_sigma;
    double w0 = S->omega0;
    const double *W1 = S->W1 + (size_t)i * Ns * 3, *b1 = S->b1 + (size_t)i * Ns, *w2 = S->w2 + (size_t)i * Ns;
    double u[3];
    for (int k = 0; k < 3; ++k) u[k] = (o[k] - P->c[k] + tm * d[k]) * P->inv_m;
    double acc = S->b2[i];
    for (int k = 0; k < Ns; ++k) {
        const double *w = W1 + 3 * k;
        double phi = w0 * (w[0] * u[0] + w[1] * u[1] + w[2] * u[2] + b1[k]) + time_phase(S, i, k);
        double th = w0 * (w[0] * d[0] + w[1] * d[1] + w[2] * d[2]) * half * P->inv_m;
        acc += w2[k] * cos(phi) * sinc(th);
    }
    return 2.0 * half * acc;
}

/* Eq. 8 literally: S(t) = sum_k w2_k / a_k sin(a_k t + psi_k) + b2 t with
 * a_k = w0 W1_k . d / m, psi_k = w0 (W1_k . (o - c) / m + b1_k) (+ xi_t W_t,k); returns S(t1) - S(t0).
 * Undefined (division by zero) when some a_k == 0. */
static double integral_naive(const ora_scene *S, int64_t i, const prim64 *P, const double o[3],
                             const double d[3], double t0, double t1)
{
    int Ns = S->n_sigma;
    double w0 = S->omega0;
    const double *W1 = S->W1 + (size_t)i * Ns * 3, *b1 = S->b1 + (size_t)i * Ns, *w2 = S->w2 + (size_t)i * Ns;
    double oc[3] = {o[0] - P->c[0], o[1] - P->c[1], o[2] - P->c[2]};
    double s0 = S->b2[i] * t0, s1 = S->b2[i] * t1;
    for (int k = 0; k < Ns; ++k) {
        const double *w = W1 + 3 * k;
        double a = w0 * (w[0] * d[0] + w[1] * d[1] + w[2] * d[2]) * P->inv_m;
        double psi = w0 * ((w[0] * oc[0] + w[1] * oc[1] + w[2] * oc[2]) * P->inv_m + b1[k]) + time_phase(S, i, k);
        s0 += w2[k] / a * sin(a * t0 + psi);
        s1 += w2[k] / a * sin(a * t1 + psi);
    }
    return s1 - s0;
}

static double relu(double x) { return x > 0.0 ? x : 0.0; }

/* The 16 real spherical harmonics of degrees 0..3 at the unit vector v = (x, y, z),
 * index l^2 + l + m, in the usual real (tesseral) form:
 *   l = 0: 1/2 sqrt(1/pi)
 *   l = 1: sqrt(3/(4 pi)) (y, z, x)
 *   l = 2: 1/2 sqrt(15/pi) xy, 1/2 sqrt(15/pi) yz, 1/4 sqrt(5/pi) (3z^2 - 1),
 *          1/2 sqrt(15/pi) xz, 1/4 sqrt(15/pi) (x^2 - y^2)
 *   l = 3: 1/4 sqrt(35/(2 pi)) y (3x^2 - y^2), 1/2 sqrt(105/pi) xyz,
 *          1/4 sqrt(21/(2 pi)) y (5z^2 - 1), 1/4 sqrt(7/pi) z (5z^2 - 3),
 *          1/4 sqrt(21/(2 pi)) x (5z^2 - 1), 1/4 sqrt(105/pi) z (x^2 - y^2),
 *          1/4 sqrt(35/(2 pi)) x (x^2 - 3y^2). */
static void sh_basis(const double v[3], double Y[16])
{
    const double pi = acos(-1.0), x = v[0], y = v[1], z = v[2];
    Y[0] = 0.5 * sqrt(1.0 / pi);
    const double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = k1 * y;
    Y[2] = k1 * z;
    Y[3] = k1 * x;
    Y[4] = 0.5 * sqrt(15.0 / pi) * x * y;
    Y[5] = 0.5 * sqrt(15.0 / pi) * y * z;
    Y[6] = 0.25 * sqrt(5.0 / pi) * (3.0 * z * z - 1.0);
    Y[7] = 0.5 * sqrt(15.0 / pi) * x * z;
    Y[8] = 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
    Y[9] = 0.25 * sqrt(35.0 / (2.0 * pi)) * y * (3.0 * x * x - y * y);
    Y[10] = 0.5 * sqrt(105.0 / pi) * x * y * z;
    Y[11] = 0.25 * sqrt(21.0 / (2.0 * pi)) * y * (5.0 * z * z - 1.0);
    Y[12] = 0.25 * sqrt(7.0 / pi) * z * (5.0 * z * z - 3.0);
    Y[13] = 0.25 * sqrt(21.0 / (2.0 * pi)) * x * (5.0 * z * z - 1.0);
    Y[14] = 0.25 * sqrt(105.0 / pi) * z * (x * x - y * y);
    Y[15] = 0.25 * sqrt(35.0 / (2.0 * pi)) * x * (x * x - 3.0 * y * y);
}

/* Colour of primitive i seen from a camera at o along the pixel's unit ray d.
 * MLP (App. D.2 colour field in the ReLU/sigmoid form): z0 = [d, f],
 * z1 = relu(Wc1 z0 + bc1), z2 = relu(Wc2 z1 + bc2), c = sigmoid(Wc3 z2 + bc3).
 * Spherical harmonics: c = max(0, 1/2 + sum_i Y_i(v) sh_i) with v the unit
 * direction from o to the primitive centre; for a time-conditioned scene the
 * degree-0 coefficient is the series sh_0 + sum_{j=1..4} a_j xi^j
 * + sum_{j=1..4} (b_j cos(j xi) + c_j sin(j xi)) (App. Applications).  Constant
 * mode returns rgb. */
static void color_eval(const ora_scene *S, int64_t i, const double o[3], const double d[3], double out[3])
{
    if (S->color_mode == ORA_COLOR_CONST) {
        for (int k = 0; k < 3; ++k) out[k] = S->rgb[3 * i + k];
        return;
    }
    if (S->color_mode == ORA_COLOR_SH) {
        const double *c = S->centers + 3 * i;
        double v[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
        const double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int k = 0; k < 3; ++k) v[k] /= nv;
        double Y[16];
        sh_basis(v, Y);
        const double *K = S->sh + (size_t)i * 48;
        for (int ch = 0; ch < 3; ++ch) {
            double a = 0.5;
            for (int b = 0; b < 16; ++b) a += Y[b] * K[3 * b + ch];
            if (S->sh_t) {
                const double *T = S->sh_t + (size_t)i * 36, x = S->time;
                double dc = 0.0;
                for (int j = 1; j <= 4; ++j)
                    dc += T[3 * (j - 1) + ch] * pow(x, j) + T[3 * (3 + j) + ch] * cos(j * x) +
                          T[3 * (7 + j) + ch] * sin(j * x);
                a += Y[0] * dc;
            }
            out[ch] = relu(a);
        }
        return;
    }
    int Nc = S->n_c, F = ORA_FEAT, fin = 3 + ORA_FEAT;
    const double *f = S->feat + (size_t)i * F;
    const double *W1c = S->Wc1 + (size_t)i * Nc * fin, *B1 = S->bc1 + (size_t)i * Nc;
    const double *W2c = S->Wc2 + (size_t)i * Nc * Nc, *B2 = S->bc2 + (size_t)i * Nc;
    const double *W3c = S->Wc3 + (size_t)i * 3 * Nc, *B3 = S->bc3 + (size_t)i * 3;
    double z0[3 + ORA_FEAT];
    for (int k = 0; k < 3; ++k) z0[k] = d[k];
    for (int k = 0; k < F; ++k) z0[3 + k] = f[k];
    double z1[256], z2[256];
    for (int j = 0; j < Nc; ++j) {
        double a = B1[j];
        for (int k = 0; k < fin; ++k) a += W1c[j * fin + k] * z0[k];
        z1[j] = relu(a);
    }
    for (int j = 0; j < Nc; ++j) {
        double a = B2[j];
        for (int k = 0; k < Nc; ++k) a += W2c[j * Nc + k] * z1[k];
        z2[j] = relu(a);
    }
    for (int r = 0; r < 3; ++r) {
        double a = B3[r];
        for (int k = 0; k < Nc; ++k) a += W3c[r * Nc + k] * z2[k];
        out[r] = 1.0 / (1.0 + exp(-a));
    }
}

/* Unit ray through the centre of pixel (px, py): d = normalize(R_wc^T ((px+.5-cx)/fx, (py+.5-cy)/fy, 1)). */
static void pixel_ray(const ora_camera *cam, int px, int py, double d[3])
{
    double x = ((double)px + 0.5 - (double)cam->cx) / (double)cam->fx;
    double y = ((double)py + 0.5 - (double)cam->cy) / (double)cam->fy;
    const float *W = cam->R_wc;
    double r[3];
    for (int k = 0; k < 3; ++k) r[k] = (double)W[0 + k] * x + (double)W[3 + k] * y + (double)W[6 + k];
    double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int k = 0; k < 3; ++k) d[k] = r[k] / nr;
}

/* Render selected pixels of one camera.
 *   pix[n_pix]        linear pixel index y * W + x
 *   pix_list[n_pix]   which candidate list each pixel walks
 *   list_off[], list_prim[]  CSR candidate lists, each already in compositing
 *                     (depth-key) order
 *   t_min             early termination: after compositing entry i stop if T_{i+1} < t_min
 *                     (t_min = 0 disables it)
 * Outputs per pixel: rgb (incl. background), tau = optical depth composited,
 * n_walk = 1 + list position of the last composited entry (0 if none), flags
 * bit 0 = a termination test landed within 1% of t_min (FP32 may decide either way).
 * Returns the number of composited pairs. */
int64_t ora_render(const ora_scene *S, const ora_camera *cam, const int32_t *pix, int64_t n_pix,
                   const int32_t *pix_list, const int64_t *list_off, const int32_t *list_prim,
                   double t_min, const double *bg, int32_t form, double *out_rgb, double *out_tau,
                   int32_t *out_nwalk, int32_t *out_flags)
{
    ora_scene St = *S; /* this view's timestamp */
    St.time = (double)cam->time;
    S = &St;
    int64_t n = S->n;
    prim64 *P = (prim64 *)malloc(sizeof(prim64) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) prim_setup(S, i, &P[i]);
    double o[3] = {cam->eye[0], cam->eye[1], cam->eye[2]};
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t p = 0; p < n_pix; ++p) {
        int px = pix[p] % cam->width, py = pix[p] / cam->width;
        double d[3];
        pixel_ray(cam, px, py, d);
        double C[3] = {0, 0, 0}, tau = 0.0, T = 1.0;
        int32_t nwalk = 0, flags = 0;
        int32_t L = pix_list[p];
        for (int64_t e = list_off[L]; e < list_off[L + 1]; ++e) {
            int64_t i = list_prim[e];
            double tm, half;
            if (!intersect(&P[i], o, d, &tm, &half)) continue;
            double ah = (form == ORA_FORM_NAIVE) ? integral_naive(S, i, &P[i], o, d, tm - half, tm + half)
                                                 : integral_stable(S, i, &P[i], o, d, tm, half);
            if (!(ah > 0.0)) continue;
            double alpha = -expm1(-ah);
            double col[3];
            color_eval(S, i, o, d, col);
            for (int k = 0; k < 3; ++k) C[k] += T * alpha * col[k];
            tau += ah;
            T = exp(-tau);
            total += 1;
            nwalk = (int32_t)(e - list_off[L] + 1);
            if (t_min > 0.0 && fabs(T - t_min) < 0.01 * t_min) flags |= 1;
            if (T < t_min) break;
        }
        for (int k = 0; k < 3; ++k) out_rgb[3 * p + k] = C[k] + T * bg[k];
        out_tau[p] = tau;
        out_nwalk[p] = nwalk;
        out_flags[p] = flags;
    }
    free(P);
    return total;
}

/* Single ray / primitive evaluation for the pins: out = {hit, t_in, t_out, alpha_hat}. */
void ora_pair(const ora_scene *S, int64_t i, const double *o, const double *d, int32_t form, double *out)
{
    prim64 P;
    prim_setup(S, i, &P);
    double tm, half;
    int hit = intersect(&P, o, d, &tm, &half);
    out[0] = hit;
    out[1] = tm - half;
    out[2] = tm + half;
    out[3] = 0.0;
    if (hit)
        out[3] = (form == ORA_FORM_NAIVE) ? integral_naive(S, i, &P, o, d, tm - half, tm + half)
                                          : integral_stable(S, i, &P, o, d, tm, half);
}

/* Integral over an arbitrary parameter interval [t0, t1] (either form). */
double ora_integral(const ora_scene *S, int64_t i, const double *o, const double *d, double t0, double t1,
                    int32_t form)
{
    prim64 P;
    prim_setup(S, i, &P);
    if (form == ORA_FORM_NAIVE) return integral_naive(S, i, &P, o, d, t0, t1);
    return integral_stable(S, i, &P, o, d, 0.5 * (t0 + t1), 0.5 * (t1 - t0));
}

void ora_color(const ora_scene *S, int64_t i, const double *o, const double *d, double *out)
{
    color_eval(S, i, o, d, out);
}

void ora_sh_basis(const double *v, double *Y) { sh_basis(v, Y); }

void ora_pixel_ray(const ora_camera *cam, int32_t px, int32_t py, double *d) { pixel_ray(cam, px, py, d); }
