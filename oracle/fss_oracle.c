/*
 * fss_oracle.c -- plain, slow FP64 reference of the 2DGS Top-K feature
 * rasterizer of Fast-SegSim (arXiv 2604.10951).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only on
 * the seeded inputs.
 *
 * What it computes, and where the paper defines it:
 *   - surfel frame and the local-to-world map (Sec. 3.1, Eq. 1);
 *   - the homogeneous surfel-to-screen transform T with rows T1, T2, Tw
 *     (Sec. 3.2, x' = T u);
 *   - the ray-splat intersection u(x): the paper names it (the pixel's
 *     projection into the surfel's tangent plane, Sec. 3.1, after Eq. 2)
 *     without a formula; it is derived here from x' = T u: the
 *     two image lines through pixel x back-project to the planes
 *     (T1 - x Tw).u = 0 and (T2 - y Tw).u = 0, whose intersection is
 *     u ~ (T1 - x Tw) x (T2 - y Tw);
 *   - the density f(u) = exp(-(u^2+v^2)/2) and front-to-back alpha
 *     compositing over depth-sorted surfels (Sec. 3.1, Eq. 2);
 *   - Top-K Hard Selection: the feature sum restricted to the K surfels of
 *     largest blending weight w_i = alpha_i * T_i (Sec. 3.4, Eq. 7); the
 *     paper's omega_i is read as the transmittance T_i;
 *   - Precise Tile Intersection: the screen conic of the cutoff disc, its
 *     tight box (SnugBox) and per-row/column extents from the quadratic
 *     A x^2 + (2B y + 2D) x + (C y^2 + 2E y + F) = 0 (AccuTile)
 *     (Sec. 3.2, the SnugBox and AccuTile subsection);
 *   - analytic gradients of the rendered outputs (the paper trains through
 *     the differentiable renderer end to end, Sec. 3.1, Sec. 3.5; it
 *     prints no gradient formulas, so the chain rule of the forward is
 *     written out directly).
 *
 * Precision: everything is double, except the tile binning, which decides
 * integers (tile lists, culling) and therefore follows the kernel's binary32
 * operation sequence exactly ("binning mirror", section 2 below).  Compile
 * with -ffp-contract=off so that no multiply-add is fused.
 *
 * Readings of silent / garbled passages (all listed in the design notes):
 *   - constants: alpha_min = 1/255, alpha_max = 0.99, T_min = 1e-4,
 *     near = 0.2 are parameters with those defaults;
 *   - sort key: the surfel centre's camera depth (binary32 bits, then index);
 *   - the printed Sigma' matrix (Sec. 3.2) is dimensionally inconsistent; the
 *     exact homography conic Q = T^-T diag(1,1,-k^2) T^-1 is used instead,
 *     which is what the printed quadratic with D, E, F requires;
 *   - k^2 = 2 ln(o / alpha_min): the cutoff where o f(u) reaches alpha_min;
 *   - stop rules: TMIN stops before a surfel that would take T below T_min;
 *     EXACT_TOPK additionally stops once the K-set is full and no later
 *     surfel can enter it (alpha_max * T <= smallest selected weight); with
 *     the first-K selection (select = 1, the other reading of Eq. 7) it
 *     stops once K surfels contributed;
 *   - Eq. 7 sums the selected w_i c_i without normalising; the variant
 *     renorm = 1 divides that sum by the selected weights' sum W_K (the
 *     selected surfels' share of the pixel becomes 1), which the paper does
 *     not use and the GPU path offers as an option.
 *
 * Borderline decisions.  Where a discrete decision of Eq. 2 / Eq. 7 (skip
 * below alpha_min, the near plane, the T_min stop, the exact Top-K stop,
 * the K-th place of the selection, the median-depth switch) is taken
 * within rounding distance of its threshold (the FLAG_* distances below),
 * a binary32 evaluation may take it the other way, and both results are
 * correct.  orc_render and orc_render_backward therefore accept a per-pixel
 * flip mask: bit b takes the b-th borderline decision of the pixel's
 * traversal (in traversal order, the selection's K-th place last) the other
 * way, and bit FLIP_MEDIAN the median-depth switch.  A zero mask is the
 * plain definition.  Nothing else changes, so each mask gives one of the
 * results a correct evaluation may produce.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* interface structs (mirrored by ctypes in oracle/__init__.py)         */
/* ------------------------------------------------------------------ */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
    float viewmat[12]; /* row-major 3x4 world->camera [R | t] */
    float near_plane;
} orc_cam;

typedef struct {
    int32_t tile_size;
    int32_t K;         /* 0: full accumulation; >0: Top-K */
    int32_t bin_mode;  /* 0 AABB, 1 SNUG, 2 ACCU */
    int32_t stop_rule; /* 0 TMIN, 1 EXACT_TOPK */
    float alpha_min, alpha_max, T_min;
    float bg[3];
    int32_t C;
    int32_t select;    /* 0: K largest weights (Eq. 7); 1: first K in depth order */
    int32_t renorm;    /* K > 0: 1 divides the Top-K sum by the selected weights' sum */
    int32_t lowpass;   /* 1: the 2DGS screen-space low-pass filter (see below) */
} orc_params;

enum { ORC_AABB = 0, ORC_SNUG = 1, ORC_ACCU = 2 };
enum { ORC_TMIN = 0, ORC_EXACT = 1 };

/* per-pixel flags: decisions taken within rounding distance of a threshold */
enum {
    FLAG_ALPHA = 1,  /* some |o f(u) - alpha_min| < 1e-6          */
    FLAG_TMIN = 2,   /* some |T (1 - alpha) - T_min| < 1e-8       */
    FLAG_TIE = 4,    /* |w_(K) - w_(K+1)| <= 1e-6                 */
    FLAG_EXACT = 8,  /* EXACT_TOPK stop within 1e-6 of its bound  */
    FLAG_NEAR = 16,  /* some |z_hit - near| < 1e-5                */
    FLAG_CLAMP = 32, /* some |o f(u) - alpha_max| < 1e-6          */
    FLAG_GRAZE = 64, /* contributor seen nearly edge-on           */
    FLAG_MEDIAN = 128, /* some |T (1 - alpha) - 1/2| < 1e-6 (median depth) */
    FLAG_LOWPASS = 256 /* low-pass: some |rho_obj - rho_screen| < 1e-3 (the derivative switches; the
                          binary32 centre moves rho_screen by up to ~1e-4 at a few pixels) */
};

#define DEG_EPS 1e-3 /* edge-on cull: |n . p_c| <= DEG_EPS |p_c| */

/* flip-mask bit of the median-depth switch; bits 0..30 are the traversal's
 * and the selection's borderline decisions in the order they are met */
#define FLIP_MEDIAN 0x80000000u

/* A decision with outcome `taken`; when `borderline` it is the next
 * borderline decision of the pixel (counted in *nb) and bit *nb of `flip`
 * takes it the other way. */
static int decide(int taken, int borderline, uint32_t flip, int *nb)
{
    if (!borderline) return taken;
    const int b = (*nb)++;
    return (b < 31 && ((flip >> b) & 1u)) ? !taken : taken;
}

/* ================================================================== */
/* 1. FP64 geometry                                                     */
/* ================================================================== */

/* Rotation of the normalised quaternion (w, x, y, z): columns t_u, t_v and
 * the normal n = t_u x t_v (Sec. 3.1). */
static void frame64(const double *q, double tu[3], double tv[3], double nrm[3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double s = sqrt(w * w + x * x + y * y + z * z);
    w /= s; x /= s; y /= s; z /= s;
    tu[0] = 1 - 2 * (y * y + z * z); tu[1] = 2 * (x * y + w * z); tu[2] = 2 * (x * z - w * y);
    tv[0] = 2 * (x * y - w * z); tv[1] = 1 - 2 * (x * x + z * z); tv[2] = 2 * (y * z + w * x);
    nrm[0] = 2 * (x * z + w * y); nrm[1] = 2 * (y * z - w * x); nrm[2] = 1 - 2 * (x * x + y * y);
}

static void matvec3(const double R[9], const double v[3], double o[3])
{
    for (int r = 0; r < 3; ++r) o[r] = R[3 * r] * v[0] + R[3 * r + 1] * v[1] + R[3 * r + 2] * v[2];
}

typedef struct {
    double T[3][3];  /* rows T1, T2, Tw */
    double pc[3];    /* surfel centre in camera space */
    double z;        /* = pc[2] */
    double cosang;   /* n.p_c / |p_c| */
    double nf[3];    /* camera-space unit normal, turned to face the camera (n.p_c <= 0) */
    double cxp, cyp; /* projected centre T (0, 0, 1) in pixels */
    int ok;          /* passes the FP64 cull rules */
} geo64;

/* T maps tangent-plane (u, v, 1) to homogeneous pixels (Sec. 3.2):
 * T = Kcam [ Rv r_u t_u | Rv r_v t_v | Rv p + t ]. */
static void geometry64(const double *mean, const double *scale, const double *quat, double opac,
                       const orc_cam *cam, const orc_params *p, geo64 *g)
{
    double R[9], t[3], tu[3], tv[3], n[3], au[3], av[3], pw[3], nc[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = cam->viewmat[4 * r + c];
        t[r] = cam->viewmat[4 * r + 3];
    }
    frame64(quat, tu, tv, n);
    matvec3(R, tu, au);
    matvec3(R, tv, av);
    matvec3(R, n, nc);
    for (int k = 0; k < 3; ++k) { au[k] *= scale[0]; av[k] *= scale[1]; pw[k] = mean[k]; }
    matvec3(R, pw, g->pc);
    for (int k = 0; k < 3; ++k) g->pc[k] += t[k];
    const double fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy;
    const double *cols[3] = {au, av, g->pc};
    for (int c = 0; c < 3; ++c) {
        g->T[0][c] = fx * cols[c][0] + cx * cols[c][2];
        g->T[1][c] = fy * cols[c][1] + cy * cols[c][2];
        g->T[2][c] = cols[c][2];
    }
    g->z = g->pc[2];
    g->cxp = g->T[0][2] / g->T[2][2];
    g->cyp = g->T[1][2] / g->T[2][2];
    double pn = sqrt(g->pc[0] * g->pc[0] + g->pc[1] * g->pc[1] + g->pc[2] * g->pc[2]);
    g->cosang = (nc[0] * g->pc[0] + nc[1] * g->pc[1] + nc[2] * g->pc[2]) / pn;
    const double sgn = g->cosang > 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < 3; ++k) g->nf[k] = sgn * nc[k];
    g->ok = (g->z > cam->near_plane) && (opac >= p->alpha_min) && (fabs(g->cosang) > DEG_EPS);
}

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Ray-splat intersection for the pixel point (x, y): returns 1 if valid. */
static int ray_splat64(const double T[3][3], double x, double y, double near,
                       double *u, double *v, double *zhit, double hx[3], double hy[3], double c[3])
{
    for (int k = 0; k < 3; ++k) { hx[k] = T[0][k] - x * T[2][k]; hy[k] = T[1][k] - y * T[2][k]; }
    cross3(hx, hy, c);
    double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (!(fabs(c[2]) > 1e-12 * cn)) return 0;
    *u = c[0] / c[2];
    *v = c[1] / c[2];
    *zhit = T[2][0] * *u + T[2][1] * *v + T[2][2];
    return *zhit > near;
}

/* ================================================================== */
/* 2. binning mirror: binary32, fixed operation order, no fused ops      */
/* ================================================================== */
/*
 * Operation-order specification (the CUDA projection kernel follows the
 * same sequence; every line is one IEEE binary32 operation, rounded to
 * nearest, evaluated left to right, no multiply-add contraction):
 *  S1  n2 = ((qw*qw + qx*qx) + qy*qy) + qz*qz; invalid unless n2 > 0;
 *      n = sqrt(n2); (w,x,y,z) = (qw/n, qx/n, qy/n, qz/n)
 *  S2  tu = (1 - 2*(y*y + z*z), 2*(x*y + w*z), 2*(x*z - w*y))
 *      tv = (2*(x*y - w*z), 1 - 2*(x*x + z*z), 2*(y*z + w*x))
 *  S3  (Rv v)_r = (R_r0*v0 + R_r1*v1) + R_r2*v2; au = su*(Rv tu);
 *      av = sv*(Rv tv); pc = (Rv p)_r + t_r
 *  S4  z = pc2; cull unless z > near
 *  S5  cull unless o >= alpha_min
 *  S5b conservative frustum test (a geometric cull like S17, placed
 *      anywhere after S5): kk = (2 * ln32(o / alpha_min)) * 1.0009765625f;
 *      rho = ((sqrt(max(kk, 0)) * max(su, sv)) * 1.001f) + 1e-6f;
 *      zlo = pc2 - rho; zhi = pc2 + rho; if zlo > 0: xa = pc0 - rho,
 *      xb = pc0 + rho (same for y); ux_max = xb / (xb >= 0 ? zlo : zhi),
 *      ux_min = xa / (xa >= 0 ? zhi : zlo) (same for y);
 *      px_max = fx*ux_max + cx, px_min = fx*ux_min + cx (same for y);
 *      cull if px_max < -0.5 or px_min > W + 0.5 or py_max < -0.5 or
 *      py_min > H + 0.5.  The sphere of radius rho about the centre holds
 *      the binning disk, so in exact arithmetic this culls only surfels
 *      whose footprint misses every pixel centre by more than a pixel.
 *  S6  k2 = 2 ln(o / alpha_min) by the binary32 procedure ln32 below:
 *      x = o / alpha_min; (m, e) = frexp(x); if m < 0.70710677f
 *      { m = m * 2; e = e - 1 }; s = (m - 1) / (m + 1); s2 = s * s;
 *      p = (((((s2 * (1/9)) + 1/7) * s2 + 1/5) * s2 + 1/3) * s2) + 1;
 *      ln x = ((float)e * 0.6931472f) + ((2 * s) * p); k2 = 2 * ln x
 *      (ln m = 2 atanh((m-1)/(m+1)), series to s^9; |s| <= 0.1716)
 *  S7  columns c_j of T for (au, av, pc):
 *      (fx*a0 + cx*a2, fy*a1 + cy*a2, a2)
 *  S8  xc = c2_0 / c2_2; yc = c2_1 / c2_2
 *  S9  shifted columns d_j = (c_j0 - xc*c_j2, c_j1 - yc*c_j2, c_j2)
 *  S10 adjugate rows m0 = d1 x d2, m1 = d2 x d0, m2 = d0 x d1, with
 *      a x b = (a1*b2 - a2*b1, a2*b0 - a0*b2, a0*b1 - a1*b0)
 *  S11 det = (d0_0*m0_0 + d0_1*m0_1) + d0_2*m0_2
 *  S12 pn = sqrt((pc0*pc0 + pc1*pc1) + pc2*pc2);
 *      cull unless |det| > 1e-3f * ((((fx*fy)*su)*sv)*pn)   (edge-on)
 *  S13 e = exponent of max|m_ij| (frexp); m_ij <- ldexp(m_ij, -e);
 *      det <- ldexp(det, -e)                       (exact rescale)
 *  S14 kb = k2 * 1.0009765625f (2^-10 relative slack);
 *      Q_ab = (m0_a*m0_b + m1_a*m1_b) - kb*(m2_a*m2_b);
 *      (A,B,C,D,E,F) = (Q00, Q01, Q11, Q02, Q12, Q22)
 *  S15 g = A*C - B*B; if !(A > 0 && g > 0): unbounded -> whole image
 *  S16 X0 = (B*E - C*D)/g; Y0 = (B*D - A*E)/g; Fp = (F + D*X0) + E*Y0;
 *      cull unless Fp < 0; hx = sqrt(((-Fp)*C)/g); hy = sqrt(((-Fp)*A)/g)
 *  S17 pixel range: px0 = ceil(((X0 - hx) + xc) - 0.5),
 *      px1 = floor(((X0 + hx) + xc) - 0.5), same for y; clamp to the image;
 *      cull if empty
 *  S18 tile rect = pixel range / ts (integer division)
 *  S19 AABB mode: square of half-size max(hx', hy') about (X0', Y0') for the
 *      opacity-blind cutoff k2' = max(kb, 2 * ln32(1 / alpha_min)),
 *      united with the S17 range
 *  S20 ACCU mode: outer loop over tile rows if (rows <= cols) else columns;
 *      per strip, extreme abscissa from the tangent point
 *      Y_L = -(B*X_L + E)/C at X_L = X0 - hx (resp. X0 + hx), else the root
 *      of the quadratic at the clamped strip edge:
 *      b = B*Y + D; c = ((C*Y)*Y + (2E)*Y) + F; disc = max(b*b - A*c, 0);
 *      x = ((-b) -/+ sqrt(disc))/A; pixel columns
 *      [ceil((x_min + xc) - 0.5), floor((x_max + xc) - 0.5)] clipped to S17.
 * Low-pass filter (lowpass = 1): the footprint also holds the screen disc
 * 2 |x - c|^2 <= k^2 about the projected centre c = (xc, yc):
 *  S5b' the S5b margins 0.5 become mg = 0.5 + sqrt(max(kk, 0) * 0.5)
 *  S17b rd2 = kb * 0.5; rd = sqrt(rd2); disc pixel range
 *      [ceil((xc - rd) - 0.5), floor((xc + rd) - 0.5)] (same for y), clamped
 *      to the image; the S17 range becomes the union of the ellipse's (when
 *      S16 keeps it and its range is not empty) and the disc's; cull only if
 *      both are empty
 *  S20b per strip [Ya, Yb] (local): Yn = Ya if Ya > 0, Yb if Yb < 0, else 0;
 *      if Yn*Yn <= rd2: hw = sqrt(rd2 - Yn*Yn), pixel columns
 *      [ceil(((-hw) + xc) - 0.5), floor((hw + xc) - 0.5)]; the strip's
 *      interval is the hull of the ellipse's and the disc's (columns alike).
 * k^2 only has to be identical on both sides (binning adds a 2^-10 slack);
 * the series is accurate to a few ulp, far inside that slack.
 */
typedef struct {
    int visible;  /* passes S1, S4, S5, S12 and the bbox is non-empty */
    int culled_by_rule;
    int unbounded;
    float z, k2, xc, yc, det;
    float m[9];
    float A, B, C, D, E, F;
    float X0, Y0, hx, hy;
    int px0, px1, py0, py1;
    int tx0, tx1, ty0, ty1;
    int ell;         /* the ellipse range is not empty (always, without the low-pass filter) */
    int lowpass;
    float rd2;       /* low-pass screen disc radius^2 (pixels) */
} mirror_rec;

/* natural logarithm of x > 0 in binary32 (S6): ln x = e ln 2 + 2 atanh(s) */
static float ln32(float x)
{
    int e;
    float m = frexpf(x, &e);
    if (m < 0.70710677f) { m = m * 2.0f; e = e - 1; }
    float num = m - 1.0f, den = m + 1.0f;
    float s = num / den;
    float s2 = s * s;
    float p = s2 * (1.0f / 9.0f);
    p = p + (1.0f / 7.0f); p = p * s2;
    p = p + (1.0f / 5.0f); p = p * s2;
    p = p + (1.0f / 3.0f); p = p * s2;
    p = p + 1.0f;
    float t = 2.0f * s;
    t = t * p;
    float el = (float)e * 0.6931472f;
    return el + t;
}

static void mvec_f(const float R[9], const float v[3], float o[3])
{
    for (int r = 0; r < 3; ++r) {
        float a = R[3 * r] * v[0];
        float b = R[3 * r + 1] * v[1];
        a = a + b;
        b = R[3 * r + 2] * v[2];
        o[r] = a + b;
    }
}

static void cross_f(const float a[3], const float b[3], float o[3])
{
    float p, q;
    p = a[1] * b[2]; q = a[2] * b[1]; o[0] = p - q;
    p = a[2] * b[0]; q = a[0] * b[2]; o[1] = p - q;
    p = a[0] * b[1]; q = a[1] * b[0]; o[2] = p - q;
}

/* ceil/floor of a pixel-centre interval [lo, hi] clipped to [0, n-1];
 * returns 0 if empty. */
static int pix_range(float lo, float hi, int n, int *a, int *b)
{
    float fl = ceilf(lo), fh = floorf(hi);
    if (!(fl <= fh)) return 0;
    if (fh < 0.0f || fl > (float)(n - 1)) return 0;
    *a = fl < 0.0f ? 0 : (int)fl;
    *b = fh > (float)(n - 1) ? n - 1 : (int)fh;
    return *a <= *b;
}

/* conic of the disc u^2+v^2 <= kk under the (rescaled) adjugate rows */
static void conic_f(const float m[9], float kk, float q[6])
{
    const int ia[6] = {0, 0, 1, 0, 1, 2}, ib[6] = {0, 1, 1, 2, 2, 2};
    for (int k = 0; k < 6; ++k) {
        int a = ia[k], b = ib[k];
        float s0 = m[a] * m[b];
        float s1 = m[3 + a] * m[3 + b];
        float s = s0 + s1;
        float t = m[6 + a] * m[6 + b];
        t = kk * t;
        q[k] = s - t;
    }
}

/* S16: centre and half extents; returns 0 if the conic is empty */
static int ellipse_f(const float q[6], float *X0, float *Y0, float *hx, float *hy)
{
    float A = q[0], B = q[1], C = q[2], D = q[3], E = q[4], F = q[5];
    float g = A * C;
    float t = B * B;
    g = g - t;
    float a1 = B * E, a2 = C * D;
    *X0 = (a1 - a2) / g;
    a1 = B * D; a2 = A * E;
    *Y0 = (a1 - a2) / g;
    float Fp = D * *X0;
    Fp = F + Fp;
    t = E * *Y0;
    Fp = Fp + t;
    if (!(Fp < 0.0f)) return 0;
    float nF = -Fp;
    t = nF * C; t = t / g; *hx = sqrtf(t);
    t = nF * A; t = t / g; *hy = sqrtf(t);
    return 1;
}

static void mirror_project(const float *mean, const float *scale, const float *quat, float o,
                           const orc_cam *cam, const orc_params *p, int mode, mirror_rec *r)
{
    memset(r, 0, sizeof(*r));
    r->culled_by_rule = 1;
    const int W = cam->width, H = cam->height, ts = p->tile_size;
    /* S1 */
    float qw = quat[0], qx = quat[1], qy = quat[2], qz = quat[3];
    float n2 = qw * qw;
    float t = qx * qx; n2 = n2 + t;
    t = qy * qy; n2 = n2 + t;
    t = qz * qz; n2 = n2 + t;
    if (!(n2 > 0.0f)) return;
    float nn = sqrtf(n2);
    float w = qw / nn, x = qx / nn, y = qy / nn, z = qz / nn;
    /* S2 */
    float tu[3], tv[3], a, b;
    a = y * y; b = z * z; a = a + b; a = 2.0f * a; tu[0] = 1.0f - a;
    a = x * y; b = w * z; a = a + b; tu[1] = 2.0f * a;
    a = x * z; b = w * y; a = a - b; tu[2] = 2.0f * a;
    a = x * y; b = w * z; a = a - b; tv[0] = 2.0f * a;
    a = x * x; b = z * z; a = a + b; a = 2.0f * a; tv[1] = 1.0f - a;
    a = y * z; b = w * x; a = a + b; tv[2] = 2.0f * a;
    /* S3 */
    float R[9], tt[3], e[3], au[3], av[3], pc[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[3 * i + j] = cam->viewmat[4 * i + j];
        tt[i] = cam->viewmat[4 * i + 3];
    }
    mvec_f(R, tu, e);
    for (int i = 0; i < 3; ++i) au[i] = scale[0] * e[i];
    mvec_f(R, tv, e);
    for (int i = 0; i < 3; ++i) av[i] = scale[1] * e[i];
    mvec_f(R, mean, e);
    for (int i = 0; i < 3; ++i) pc[i] = e[i] + tt[i];
    /* S4, S5 */
    r->z = pc[2];
    if (!(pc[2] > cam->near_plane)) return;
    if (!(o >= p->alpha_min)) return;
    /* S6 */
    r->k2 = 2.0f * ln32(o / p->alpha_min);
    /* S7 */
    float c[3][3];
    const float *src[3] = {au, av, pc};
    for (int j = 0; j < 3; ++j) {
        a = cam->fx * src[j][0]; b = cam->cx * src[j][2]; c[j][0] = a + b;
        a = cam->fy * src[j][1]; b = cam->cy * src[j][2]; c[j][1] = a + b;
        c[j][2] = src[j][2];
    }
    /* S8 */
    r->xc = c[2][0] / c[2][2];
    r->yc = c[2][1] / c[2][2];
    /* S9 */
    float d[3][3];
    for (int j = 0; j < 3; ++j) {
        a = r->xc * c[j][2]; d[j][0] = c[j][0] - a;
        a = r->yc * c[j][2]; d[j][1] = c[j][1] - a;
        d[j][2] = c[j][2];
    }
    /* S10 */
    cross_f(d[1], d[2], &r->m[0]);
    cross_f(d[2], d[0], &r->m[3]);
    cross_f(d[0], d[1], &r->m[6]);
    /* S11 */
    a = d[0][0] * r->m[0]; b = d[0][1] * r->m[1]; a = a + b;
    b = d[0][2] * r->m[2]; float det = a + b;
    /* S12 */
    a = pc[0] * pc[0]; b = pc[1] * pc[1]; a = a + b; b = pc[2] * pc[2]; a = a + b;
    float pn = sqrtf(a);
    float lim = cam->fx * cam->fy;
    lim = lim * scale[0]; lim = lim * scale[1]; lim = lim * pn; lim = 1e-3f * lim;
    if (!(fabsf(det) > lim)) return;
    /* S13 */
    float mx = 0.0f;
    for (int i = 0; i < 9; ++i) mx = fabsf(r->m[i]) > mx ? fabsf(r->m[i]) : mx;
    if (!(mx > 0.0f)) return;
    int ex;
    frexpf(mx, &ex);
    for (int i = 0; i < 9; ++i) r->m[i] = ldexpf(r->m[i], -ex);
    r->det = ldexpf(det, -ex);
    r->culled_by_rule = 0;
    /* S5b */
    {
        float kk = o / p->alpha_min;
        kk = ln32(kk); kk = 2.0f * kk; kk = kk * 1.0009765625f;
        float rho = sqrtf(fmaxf(kk, 0.0f));
        rho = rho * fmaxf(scale[0], scale[1]); rho = rho * 1.001f; rho = rho + 1e-6f;
        const float zlo = pc[2] - rho, zhi = pc[2] + rho;
        if (zlo > 0.0f) {
            const float xa = pc[0] - rho, xb = pc[0] + rho, ya = pc[1] - rho, yb = pc[1] + rho;
            const float uxmax = xb / (xb >= 0.0f ? zlo : zhi), uxmin = xa / (xa >= 0.0f ? zhi : zlo);
            const float uymax = yb / (yb >= 0.0f ? zlo : zhi), uymin = ya / (ya >= 0.0f ? zhi : zlo);
            a = cam->fx * uxmax; const float pxmax = a + cam->cx;
            a = cam->fx * uxmin; const float pxmin = a + cam->cx;
            a = cam->fy * uymax; const float pymax = a + cam->cy;
            a = cam->fy * uymin; const float pymin = a + cam->cy;
            float mg = 0.5f;
            if (p->lowpass) { /* S5b' */
                float rk = fmaxf(kk, 0.0f); rk = rk * 0.5f; rk = sqrtf(rk); mg = mg + rk;
            }
            if (pxmax < -mg || pxmin > (float)W + mg || pymax < -mg || pymin > (float)H + mg) return;
        }
    }
    /* S14 */
    float kb = r->k2 * 1.0009765625f;
    float q[6];
    conic_f(r->m, kb, q);
    r->A = q[0]; r->B = q[1]; r->C = q[2]; r->D = q[3]; r->E = q[4]; r->F = q[5];
    /* S15 */
    a = q[0] * q[2]; b = q[1] * q[1]; a = a - b;
    r->lowpass = p->lowpass;
    if (!(q[0] > 0.0f && a > 0.0f)) {
        r->unbounded = 1;
        r->px0 = 0; r->px1 = W - 1; r->py0 = 0; r->py1 = H - 1;
    } else {
        /* S16, S17 */
        int e0 = 0, e1 = 0, f0 = 0, f1 = 0;
        r->ell = ellipse_f(q, &r->X0, &r->Y0, &r->hx, &r->hy);
        if (r->ell) {
            float lo, hi;
            lo = r->X0 - r->hx; lo = lo + r->xc; lo = lo - 0.5f;
            hi = r->X0 + r->hx; hi = hi + r->xc; hi = hi - 0.5f;
            r->ell = pix_range(lo, hi, W, &e0, &e1);
            lo = r->Y0 - r->hy; lo = lo + r->yc; lo = lo - 0.5f;
            hi = r->Y0 + r->hy; hi = hi + r->yc; hi = hi - 0.5f;
            r->ell = r->ell && pix_range(lo, hi, H, &f0, &f1);
        }
        int disc = 0, g0 = 0, g1 = 0, h0 = 0, h1 = 0;
        if (p->lowpass) { /* S17b */
            r->rd2 = kb * 0.5f;
            const float rd = sqrtf(r->rd2);
            float lo, hi;
            lo = r->xc - rd; lo = lo - 0.5f; hi = r->xc + rd; hi = hi - 0.5f;
            disc = pix_range(lo, hi, W, &g0, &g1);
            lo = r->yc - rd; lo = lo - 0.5f; hi = r->yc + rd; hi = hi - 0.5f;
            disc = disc && pix_range(lo, hi, H, &h0, &h1);
        }
        if (!r->ell && !disc) return;
        if (r->ell && disc) {
            r->px0 = e0 < g0 ? e0 : g0; r->px1 = e1 > g1 ? e1 : g1;
            r->py0 = f0 < h0 ? f0 : h0; r->py1 = f1 > h1 ? f1 : h1;
        } else if (r->ell) {
            r->px0 = e0; r->px1 = e1; r->py0 = f0; r->py1 = f1;
        } else {
            r->px0 = g0; r->px1 = g1; r->py0 = h0; r->py1 = h1;
        }
    }
    r->visible = 1;
    /* S18 */
    r->tx0 = r->px0 / ts; r->tx1 = r->px1 / ts;
    r->ty0 = r->py0 / ts; r->ty1 = r->py1 / ts;
    /* S19 */
    if (mode == ORC_AABB && !r->unbounded) {
        float k2a = 2.0f * ln32(1.0f / p->alpha_min);
        if (kb > k2a) k2a = kb;
        float qa[6], X0, Y0, hx, hy;
        conic_f(r->m, k2a, qa);
        a = qa[0] * qa[2]; b = qa[1] * qa[1]; a = a - b;
        int ax0 = 0, ax1 = W - 1, ay0 = 0, ay1 = H - 1;
        if (qa[0] > 0.0f && a > 0.0f && ellipse_f(qa, &X0, &Y0, &hx, &hy)) {
            float h = hx > hy ? hx : hy, lo, hi;
            lo = X0 - h; lo = lo + r->xc; lo = lo - 0.5f;
            hi = X0 + h; hi = hi + r->xc; hi = hi - 0.5f;
            if (!pix_range(lo, hi, W, &ax0, &ax1)) { ax0 = r->px0; ax1 = r->px1; }
            lo = Y0 - h; lo = lo + r->yc; lo = lo - 0.5f;
            hi = Y0 + h; hi = hi + r->yc; hi = hi - 0.5f;
            if (!pix_range(lo, hi, H, &ay0, &ay1)) { ay0 = r->py0; ay1 = r->py1; }
        }
        ax0 = ax0 < r->px0 ? ax0 : r->px0; ax1 = ax1 > r->px1 ? ax1 : r->px1;
        ay0 = ay0 < r->py0 ? ay0 : r->py0; ay1 = ay1 > r->py1 ? ay1 : r->py1;
        r->tx0 = ax0 / ts; r->tx1 = ax1 / ts;
        r->ty0 = ay0 / ts; r->ty1 = ay1 / ts;
    }
}

/* S20b: pixel interval [*a, *b] (clipped to [lo_clip, hi_clip]) of the
 * screen disc of radius^2 rd2 about the local origin on the strip [Sa, Sb]
 * of the other coordinate; *a > *b when it misses the strip */
static void disc_strip(float rd2, float Sa, float Sb, float origin, int lo_clip, int hi_clip, int *a, int *b)
{
    *a = 1; *b = 0;
    float Sn = Sa > 0.0f ? Sa : (Sb < 0.0f ? Sb : 0.0f);
    float s2 = Sn * Sn;
    if (!(s2 <= rd2)) return;
    float t = rd2 - s2;
    float hw = sqrtf(t);
    float lo = -hw; lo = lo + origin; lo = lo - 0.5f;
    float hi = hw + origin; hi = hi - 0.5f;
    float fl = ceilf(lo), fh = floorf(hi);
    if (!(fl <= fh) || fh < (float)lo_clip || fl > (float)hi_clip) return;
    *a = fl < (float)lo_clip ? lo_clip : (int)fl;
    *b = fh > (float)hi_clip ? hi_clip : (int)fh;
}

/* S20, outer loop over tile rows: tile-column interval of row ty */
static int accu_row(const mirror_rec *r, int ts, int ty, int *ta, int *tb)
{
    int ra = ty * ts > r->py0 ? ty * ts : r->py0;
    int rb = ty * ts + ts - 1 < r->py1 ? ty * ts + ts - 1 : r->py1;
    if (ra > rb) return 0;
    const float A = r->A, B = r->B, C = r->C, D = r->D, E = r->E, F = r->F;
    float Ya = (float)ra + 0.5f; Ya = Ya - r->yc;
    float Yb = (float)rb + 0.5f; Yb = Yb - r->yc;
    int da = 0, db = -1; /* S20b: the disc's pixel columns on this strip */
    if (r->lowpass) disc_strip(r->rd2, Ya, Yb, r->xc, r->px0, r->px1, &da, &db);
    if (!r->ell) {
        if (da > db) return 0;
        *ta = da / ts; *tb = db / ts;
        return 1;
    }
    float ext[2];
    for (int side = 0; side < 2; ++side) {
        float Xs = side == 0 ? r->X0 - r->hx : r->X0 + r->hx;
        float t = B * Xs; t = t + E; float Yt = -t / C;
        if (Yt >= Ya && Yt <= Yb) { ext[side] = Xs; continue; }
        float Y = Yt < Ya ? Ya : Yb;
        float bb = B * Y; bb = bb + D;
        float cc = C * Y; cc = cc * Y;
        float e2 = 2.0f * E; e2 = e2 * Y; cc = cc + e2; cc = cc + F;
        float disc = bb * bb; t = A * cc; disc = disc - t;
        if (disc < 0.0f) disc = 0.0f;
        float sq = sqrtf(disc);
        float nb = -bb;
        float num = side == 0 ? nb - sq : nb + sq;
        ext[side] = num / A;
    }
    float lo = ext[0] + r->xc; lo = lo - 0.5f;
    float hi = ext[1] + r->xc; hi = hi - 0.5f;
    float fl = ceilf(lo), fh = floorf(hi);
    int a = 1, b = 0;
    if (fl <= fh && !(fh < (float)r->px0 || fl > (float)r->px1)) {
        a = fl < (float)r->px0 ? r->px0 : (int)fl;
        b = fh > (float)r->px1 ? r->px1 : (int)fh;
    }
    if (da <= db) {
        if (a > b) { a = da; b = db; }
        else { a = a < da ? a : da; b = b > db ? b : db; }
    }
    if (a > b) return 0;
    *ta = a / ts; *tb = b / ts;
    return 1;
}

/* S20, outer loop over tile columns: tile-row interval of column tx */
static int accu_col(const mirror_rec *r, int ts, int tx, int *ta, int *tb)
{
    int ca = tx * ts > r->px0 ? tx * ts : r->px0;
    int cb = tx * ts + ts - 1 < r->px1 ? tx * ts + ts - 1 : r->px1;
    if (ca > cb) return 0;
    const float A = r->A, B = r->B, C = r->C, D = r->D, E = r->E, F = r->F;
    float Xa = (float)ca + 0.5f; Xa = Xa - r->xc;
    float Xb = (float)cb + 0.5f; Xb = Xb - r->xc;
    int da = 0, db = -1; /* S20b: the disc's pixel rows on this strip */
    if (r->lowpass) disc_strip(r->rd2, Xa, Xb, r->yc, r->py0, r->py1, &da, &db);
    if (!r->ell) {
        if (da > db) return 0;
        *ta = da / ts; *tb = db / ts;
        return 1;
    }
    float ext[2];
    for (int side = 0; side < 2; ++side) {
        float Ys = side == 0 ? r->Y0 - r->hy : r->Y0 + r->hy;
        float t = B * Ys; t = t + D; float Xt = -t / A;
        if (Xt >= Xa && Xt <= Xb) { ext[side] = Ys; continue; }
        float X = Xt < Xa ? Xa : Xb;
        float bb = B * X; bb = bb + E;
        float cc = A * X; cc = cc * X;
        float d2 = 2.0f * D; d2 = d2 * X; cc = cc + d2; cc = cc + F;
        float disc = bb * bb; t = C * cc; disc = disc - t;
        if (disc < 0.0f) disc = 0.0f;
        float sq = sqrtf(disc);
        float nb = -bb;
        float num = side == 0 ? nb - sq : nb + sq;
        ext[side] = num / C;
    }
    float lo = ext[0] + r->yc; lo = lo - 0.5f;
    float hi = ext[1] + r->yc; hi = hi - 0.5f;
    float fl = ceilf(lo), fh = floorf(hi);
    int a = 1, b = 0;
    if (fl <= fh && !(fh < (float)r->py0 || fl > (float)r->py1)) {
        a = fl < (float)r->py0 ? r->py0 : (int)fl;
        b = fh > (float)r->py1 ? r->py1 : (int)fh;
    }
    if (da <= db) {
        if (a > b) { a = da; b = db; }
        else { a = a < da ? a : da; b = b > db ? b : db; }
    }
    if (a > b) return 0;
    *ta = a / ts; *tb = b / ts;
    return 1;
}

/* Enumerate the tiles of one surfel (row-major order); returns the count and
 * writes up to cap tile ids into out (may be NULL). */
static int64_t tiles_of(const mirror_rec *r, const orc_cam *cam, const orc_params *p, int mode,
                        int32_t *out, int64_t cap)
{
    if (!r->visible) return 0;
    const int ts = p->tile_size, tiles_x = (cam->width + ts - 1) / ts;
    int64_t n = 0;
#define EMIT(TX, TY) do { if (out && n < cap) out[n] = (TY) * tiles_x + (TX); ++n; } while (0)
    if (mode != ORC_ACCU || r->unbounded) {
        for (int ty = r->ty0; ty <= r->ty1; ++ty)
            for (int tx = r->tx0; tx <= r->tx1; ++tx) EMIT(tx, ty);
        return n;
    }
    const int xs = r->tx1 - r->tx0 + 1, ys = r->ty1 - r->ty0 + 1;
    if (ys <= xs) {
        for (int ty = r->ty0; ty <= r->ty1; ++ty) {
            int a, b;
            if (!accu_row(r, ts, ty, &a, &b)) continue;
            for (int tx = a; tx <= b; ++tx) EMIT(tx, ty);
        }
    } else {
        /* column traversal, emitted row-major for a canonical order */
        int *lo = (int *)malloc(sizeof(int) * (size_t)xs), *hi = (int *)malloc(sizeof(int) * (size_t)xs);
        for (int tx = r->tx0; tx <= r->tx1; ++tx) {
            int a, b;
            if (!accu_col(r, ts, tx, &a, &b)) { lo[tx - r->tx0] = 1; hi[tx - r->tx0] = 0; continue; }
            lo[tx - r->tx0] = a; hi[tx - r->tx0] = b;
        }
        for (int ty = r->ty0; ty <= r->ty1; ++ty)
            for (int tx = r->tx0; tx <= r->tx1; ++tx)
                if (ty >= lo[tx - r->tx0] && ty <= hi[tx - r->tx0]) EMIT(tx, ty);
        free(lo); free(hi);
    }
#undef EMIT
    return n;
}

/* ------------------------------------------------------------------ */
/* exported: mirror records, binning, sort, ranges                       */
/* ------------------------------------------------------------------ */

/* Per-surfel mirror record: recf[N][26] = z, k2, xc, yc, det, m[9], A..F,
 * X0, Y0, hx, hy; reci[N][11] = visible, culled_by_rule, unbounded,
 * px0, px1, py0, py1, tx0, tx1, ty0, ty1; count[N] tiles in `mode`. */
void orc_mirror_project(int64_t N, const float *means, const float *scales, const float *quats,
                        const float *opac, const orc_cam *cam, const orc_params *p, int mode,
                        float *recf, int32_t *reci, int32_t *count)
{
    for (int64_t i = 0; i < N; ++i) {
        mirror_rec r;
        mirror_project(means + 3 * i, scales + 2 * i, quats + 4 * i, opac[i], cam, p, mode, &r);
        if (recf) {
            float *f = recf + 26 * i;
            f[0] = r.z; f[1] = r.k2; f[2] = r.xc; f[3] = r.yc; f[4] = r.det;
            for (int k = 0; k < 9; ++k) f[5 + k] = r.m[k];
            f[14] = r.A; f[15] = r.B; f[16] = r.C; f[17] = r.D; f[18] = r.E; f[19] = r.F;
            f[20] = r.X0; f[21] = r.Y0; f[22] = r.hx; f[23] = r.hy; f[24] = 0; f[25] = 0;
        }
        if (reci) {
            int32_t *q = reci + 11 * i;
            q[0] = r.visible; q[1] = r.culled_by_rule; q[2] = r.unbounded;
            q[3] = r.px0; q[4] = r.px1; q[5] = r.py0; q[6] = r.py1;
            q[7] = r.tx0; q[8] = r.tx1; q[9] = r.ty0; q[10] = r.ty1;
        }
        if (count) count[i] = (int32_t)tiles_of(&r, cam, p, mode, NULL, 0);
    }
}

/* Tile-surfel pairs in surfel order (tiles row-major per surfel); returns
 * the total P and writes min(P, cap) pairs. */
int64_t orc_bin(int64_t N, const float *means, const float *scales, const float *quats,
                const float *opac, const orc_cam *cam, const orc_params *p, int mode,
                int64_t cap, int32_t *pair_tile, int32_t *pair_id)
{
    int64_t P = 0;
    for (int64_t i = 0; i < N; ++i) {
        mirror_rec r;
        mirror_project(means + 3 * i, scales + 2 * i, quats + 4 * i, opac[i], cam, p, mode, &r);
        int64_t room = cap > P ? cap - P : 0;
        int64_t n = tiles_of(&r, cam, p, mode, pair_tile ? pair_tile + P : NULL, room);
        if (pair_id)
            for (int64_t k = 0; k < n && P + k < cap; ++k) pair_id[P + k] = (int32_t)i;
        P += n;
    }
    return P;
}

static const float *g_sort_z;
static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

typedef struct { int32_t tile, id; } pair_t;

static int pair_cmp(const void *pa, const void *pb)
{
    const pair_t *a = (const pair_t *)pa, *b = (const pair_t *)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    uint32_t za = fbits(g_sort_z[a->id]), zb = fbits(g_sort_z[b->id]);
    if (za != zb) return za < zb ? -1 : 1;
    return a->id < b->id ? -1 : (a->id > b->id);
}

/* Order pairs by (tile, binary32 bits of the surfel depth, surfel index)
 * (the depth order of the compositing, Sec. 3.1).  Depths are positive, so the bit
 * order is the numeric order. */
void orc_sort_pairs(int64_t P, const int32_t *tiles, const int32_t *ids, const float *z,
                    int32_t *out_tiles, int32_t *out_ids)
{
    pair_t *v = (pair_t *)malloc(sizeof(pair_t) * (size_t)(P > 0 ? P : 1));
    for (int64_t i = 0; i < P; ++i) { v[i].tile = tiles[i]; v[i].id = ids[i]; }
    g_sort_z = z;
    qsort(v, (size_t)P, sizeof(pair_t), pair_cmp);
    for (int64_t i = 0; i < P; ++i) { out_tiles[i] = v[i].tile; out_ids[i] = v[i].id; }
    free(v);
}

/* ranges[t] = [start, end) of tile t in the sorted pair list */
void orc_ranges(int64_t P, const int32_t *sorted_tiles, int32_t n_tiles, int32_t *ranges)
{
    for (int32_t t = 0; t < n_tiles; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t i = 0; i < P; ++i) {
        int32_t t = sorted_tiles[i];
        if (i == 0 || sorted_tiles[i - 1] != t) ranges[2 * t] = (int32_t)i;
        if (i == P - 1 || sorted_tiles[i + 1] != t) ranges[2 * t + 1] = (int32_t)(i + 1);
    }
}

/* ================================================================== */
/* 3. FP64 compositing (Eq. 2) with Top-K Hard Selection (Eq. 7)         */
/* ================================================================== */

typedef struct {
    int32_t pos;    /* position in the traversed list */
    int32_t id;     /* surfel index */
    double alpha, T, w;
    double u, v, oG; /* for gradients */
    double zh;       /* camera depth of the ray-surfel hit (low-pass screen term: of the centre) */
    double hx[3], hy[3], c[3];
    int scr;         /* low-pass: the screen-space term gave alpha */
    double sx, sy;   /* pixel point minus the projected centre */
} contrib_t;

typedef struct {
    double rgb[3], T;
    int32_t n_contrib, n_stop, flags;
    int32_t nsel;
    int32_t sel[32];     /* indices into the contributor array, front-to-back */
    int64_t n_eval;
    int32_t nborder;     /* borderline decisions met (traversal and selection) */
} pix_out;

/* K largest weights, ties to the earlier position (Eq. 7 set definition). */
static int wt_before(const contrib_t *a, const contrib_t *b)
{
    return a->w > b->w || (a->w == b->w && a->pos < b->pos);
}

static int cmp_int(const void *a, const void *b) { return *(const int *)a - *(const int *)b; }

/* Composite one pixel over the candidate list `cand` (surfel indices in
 * depth order); contributors are written to `cb` (capacity n_cand).
 * `flip` takes borderline decisions the other way (see decide()). */
static void composite_pixel(const geo64 *geo, const double *opac, const double *rgb, const orc_cam *cam,
                            const orc_params *p, const int32_t *cand, int32_t n_cand, double px, double py,
                            uint32_t flip, contrib_t *cb, pix_out *out)
{
    int nb = 0;
    const double amin = p->alpha_min, amax = p->alpha_max, tmin = p->T_min;
    const int K = p->K;
    double T = 1.0, rgbacc[3] = {0, 0, 0};
    int n = 0, flags = 0, n_stop = 0;
    /* running K-th largest weight for the EXACT_TOPK stop */
    double topw[33];
    int ntop = 0;
    int64_t n_eval = 0;
    for (int32_t j = 0; j < n_cand; ++j) {
        /* first-K selection: the set is final once K surfels contributed */
        if (K > 0 && p->stop_rule == ORC_EXACT && p->select == 1 && n == K) break;
        const int32_t id = cand[j];
        const geo64 *g = &geo[id];
        double u = 0.0, v = 0.0, zh = 0.0, hx[3], hy[3], c[3];
        ++n_eval;
        const int obj = ray_splat64(g->T, px, py, -INFINITY, &u, &v, &zh, hx, hy, c);
        double rho = obj ? u * u + v * v : INFINITY;
        int scr = 0;
        const double sx = px - g->cxp, sy = py - g->cyp;
        if (p->lowpass) {
            /* 2DGS low-pass filter: the larger of the object-space Gaussian and
             * a screen-space one of variance 1/2 pixel^2 about the projected
             * centre, rho = min(u^2 + v^2, 2 |x - c|^2); the screen term takes
             * the centre's depth */
            const double rs = 2.0 * (sx * sx + sy * sy);
            if (obj && fabs(rho - rs) < 1e-3) flags |= FLAG_LOWPASS;
            if (!(rho <= rs)) { rho = rs; zh = g->z; scr = 1; }
        } else if (!obj) {
            continue;
        }
        const int bnear = fabs(zh - cam->near_plane) < 1e-5;
        if (bnear) flags |= FLAG_NEAR;
        if (decide(!(zh > cam->near_plane), bnear, flip, &nb)) continue;
        double oG = opac[id] * exp(-0.5 * rho);
        const int balpha = fabs(oG - amin) < 1e-6;
        if (balpha) flags |= FLAG_ALPHA;
        if (fabs(oG - amax) < 1e-6) flags |= FLAG_CLAMP;
        double alpha = oG < amax ? oG : amax;
        if (decide(alpha < amin, balpha, flip, &nb)) continue;
        double Tn = T * (1.0 - alpha);
        const int btmin = fabs(Tn - tmin) < 1e-8;
        if (btmin) flags |= FLAG_TMIN;
        if (fabs(Tn - 0.5) < 1e-6) flags |= FLAG_MEDIAN;
        if (decide(Tn < tmin, btmin, flip, &nb)) break;
        contrib_t *e = &cb[n++];
        e->pos = j; e->id = id; e->alpha = alpha; e->T = T; e->w = alpha * T;
        e->u = u; e->v = v; e->oG = oG; e->zh = zh;
        e->scr = scr; e->sx = sx; e->sy = sy;
        memcpy(e->hx, hx, sizeof hx); memcpy(e->hy, hy, sizeof hy); memcpy(e->c, c, sizeof c);
        if (fabs(g->cosang) < 2e-3) flags |= FLAG_GRAZE;
        for (int k = 0; k < 3; ++k) rgbacc[k] += e->w * rgb[3 * id + k];
        T = Tn;
        n_stop = j + 1;
        if (K > 0) { /* running K largest weights, descending */
            int q = -1;
            if (ntop < K) q = ntop++;
            else if (e->w > topw[K - 1]) q = K - 1;
            if (q >= 0) {
                while (q > 0 && topw[q - 1] < e->w) { topw[q] = topw[q - 1]; --q; }
                topw[q] = e->w;
            }
        }
        /* EXACT_TOPK stop: once the set is full, no later surfel can enter it when
         * alpha_max T <= the smallest selected weight.  T and the set change only at a
         * contribution, so the test is taken once per contribution (one decision,
         * whatever number of candidates follow before the next contribution). */
        if (K > 0 && p->stop_rule == ORC_EXACT && p->select == 0 && ntop == K) {
            const double wmin = topw[K - 1];
            const int border = fabs(amax * T - wmin) <= 1e-6;
            if (border) flags |= FLAG_EXACT;
            if (decide(amax * T <= wmin, border, flip, &nb)) break;
        }
    }
    for (int k = 0; k < 3; ++k) out->rgb[k] = rgbacc[k] + T * p->bg[k];
    out->T = T;
    out->n_contrib = n;
    out->n_stop = n_stop;
    out->n_eval = n_eval;
    out->nsel = 0;
    if (K > 0) {
        int *idx = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
        for (int i = 0; i < n; ++i) idx[i] = i;
        int nsel = n < K ? n : K;
        if (p->select == 0) {
            /* partial selection sort by (w desc, pos asc) */
            for (int a = 0; a < nsel; ++a) {
                int best = a;
                for (int b = a + 1; b < n; ++b)
                    if (wt_before(&cb[idx[b]], &cb[idx[best]])) best = b;
                int tmp = idx[a]; idx[a] = idx[best]; idx[best] = tmp;
            }
            if (n > K) {
                /* the K-th place against the best weight left out (ties to the earlier position) */
                double wk = cb[idx[K - 1]].w, wbest_out = -1.0;
                int bout = -1;
                for (int b = K; b < n; ++b)
                    if (bout < 0 || wt_before(&cb[idx[b]], &cb[idx[bout]])) { bout = b; wbest_out = cb[idx[b]].w; }
                const int btie = fabs(wk - wbest_out) <= 1e-6;
                if (btie) flags |= FLAG_TIE;
                if (decide(0, btie, flip, &nb)) { int tmp = idx[K - 1]; idx[K - 1] = idx[bout]; idx[bout] = tmp; }
            }
        }
        qsort(idx, (size_t)nsel, sizeof(int), cmp_int); /* front-to-back */
        for (int a = 0; a < nsel; ++a) out->sel[a] = idx[a];
        out->nsel = nsel;
        free(idx);
    }
    out->flags = flags;
    out->nborder = nb;
}

/* Candidate order for the brute-force renderer: every surfel that passes
 * the cull, ascending by (binary32 depth bits, index). */
static const float *g_key;
static int key_cmp(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    uint32_t za = fbits(g_key[a]), zb = fbits(g_key[b]);
    if (za != zb) return za < zb ? -1 : 1;
    return a < b ? -1 : (a > b);
}

typedef struct {
    geo64 *geo;
    int32_t *order;
    int32_t n_order;
} scene_prep;

static void prepare(int64_t N, const double *means, const double *scales, const double *quats,
                    const double *opac, const orc_cam *cam, const orc_params *p,
                    const int32_t *visible, const float *zkey, int want_order, scene_prep *sp)
{
    sp->geo = (geo64 *)malloc(sizeof(geo64) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        geometry64(means + 3 * i, scales + 2 * i, quats + 4 * i, opac[i], cam, p, &sp->geo[i]);
        if (visible) sp->geo[i].ok = visible[i] != 0;
    }
    sp->order = NULL;
    sp->n_order = 0;
    if (want_order) {
        float *key = (float *)malloc(sizeof(float) * (size_t)(N > 0 ? N : 1));
        sp->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
        for (int64_t i = 0; i < N; ++i) {
            key[i] = zkey ? zkey[i] : (float)sp->geo[i].z;
            if (sp->geo[i].ok) sp->order[sp->n_order++] = (int32_t)i;
        }
        g_key = key;
        qsort(sp->order, (size_t)sp->n_order, sizeof(int32_t), key_cmp);
        free(key);
    }
}

static void release(scene_prep *sp) { free(sp->geo); free(sp->order); }

/*
 * Render one view.  Tiled if `ranges` is given (the sorted pair lists of a
 * binning), otherwise brute force over all surfels that pass the cull
 * (`visible` overrides the FP64 cull rules; `zkey` overrides the sort key).
 * Outputs (row-major pixels, any may be NULL):
 *   F[H*W*C], rgb[H*W*3], T[H*W], ids[H*W*K] (front-to-back, -1 padded),
 *   w[H*W*K], pos[H*W*K] (list position), nstop[H*W], ncontrib[H*W],
 *   flags[H*W]; counters[2] = (evaluations, contributions).
 * flip[H*W] (may be NULL): per-pixel flip masks of the borderline decisions
 * (see decide()); only[H*W] (may be NULL): render just the pixels where it
 * is non-zero and leave the others' outputs untouched; nborder[H*W]: the
 * borderline decisions each pixel met (the median switch not counted).
 */
void orc_render(int64_t N, const double *means, const double *scales, const double *quats,
                const double *opac, const double *rgb, const double *feats, const orc_cam *cam,
                const orc_params *p, const int32_t *ranges, const int32_t *sorted_ids,
                const int32_t *visible, const float *zkey,
                double *F, double *out_rgb, double *out_T, int32_t *ids, double *wout, int32_t *pos,
                int32_t *nstop, int32_t *ncontrib, int32_t *flags, int64_t *counters, int n_threads,
                double *depth, double *depth_med, double *normal,
                const uint32_t *flip, const uint8_t *only, int32_t *nborder)
{
    const int W = cam->width, H = cam->height, ts = p->tile_size, C = p->C, K = p->K;
    const int tiles_x = (W + ts - 1) / ts;
    scene_prep sp;
    prepare(N, means, scales, quats, opac, cam, p, visible, zkey, ranges == NULL, &sp);
    int64_t n_eval = 0, n_contrib = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_eval, n_contrib)
    for (int py = 0; py < H; ++py) {
        int64_t cap = ranges ? 0 : sp.n_order;
        if (ranges)
            for (int tx = 0; tx < tiles_x; ++tx) {
                int t = (py / ts) * tiles_x + tx;
                int64_t len = ranges[2 * t + 1] - ranges[2 * t];
                if (len > cap) cap = len;
            }
        contrib_t *cb = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(cap > 0 ? cap : 1));
        for (int px = 0; px < W; ++px) {
            const int32_t *cand;
            int32_t n_cand;
            if (ranges) {
                int t = (py / ts) * tiles_x + px / ts;
                cand = sorted_ids + ranges[2 * t];
                n_cand = ranges[2 * t + 1] - ranges[2 * t];
            } else {
                cand = sp.order;
                n_cand = sp.n_order;
            }
            const int64_t pix = (int64_t)py * W + px;
            if (only && !only[pix]) continue;
            const uint32_t fl = flip ? flip[pix] : 0u;
            pix_out o;
            composite_pixel(sp.geo, opac, rgb, cam, p, cand, n_cand, px + 0.5, py + 0.5, fl, cb, &o);
            if (nborder) nborder[pix] = o.nborder;
            n_eval += o.n_eval;
            n_contrib += o.n_contrib;
            if (out_rgb) for (int k = 0; k < 3; ++k) out_rgb[3 * pix + k] = o.rgb[k];
            if (out_T) out_T[pix] = o.T;
            if (nstop) nstop[pix] = o.n_stop;
            if (ncontrib) ncontrib[pix] = o.n_contrib;
            if (flags) flags[pix] = o.flags;
            /* sensor outputs over the traversed contributors, like RGB: expected
             * depth sum w z_hit, median depth (the hit where T first drops below
             * 1/2, else 0) and normal sum w n (camera space, facing the camera) */
            if (depth || depth_med || normal) {
                double dz = 0.0, zm = 0.0, nn[3] = {0.0, 0.0, 0.0};
                int found = 0;
                for (int i = 0; i < o.n_contrib; ++i) {
                    const contrib_t *e = &cb[i];
                    dz += e->w * e->zh;
                    for (int k = 0; k < 3; ++k) nn[k] += e->w * sp.geo[e->id].nf[k];
                    if (found) continue;
                    const double Tn = e->T * (1.0 - e->alpha);
                    /* the switch within rounding distance of 1/2 may go the other way */
                    const int below = Tn < 0.5;
                    if ((fabs(Tn - 0.5) < 1e-6 && (fl & FLIP_MEDIAN)) ? !below : below) { zm = e->zh; found = 1; }
                }
                if (depth) depth[pix] = dz;
                if (depth_med) depth_med[pix] = zm;
                if (normal) for (int k = 0; k < 3; ++k) normal[3 * pix + k] = nn[k];
            }
            if (F) {
                double *f = F + pix * C;
                for (int ch = 0; ch < C; ++ch) f[ch] = 0.0;
                if (K == 0) {
                    for (int i = 0; i < o.n_contrib; ++i) {
                        const double *c = feats + (int64_t)cb[i].id * C;
                        for (int ch = 0; ch < C; ++ch) f[ch] += cb[i].w * c[ch];
                    }
                } else {
                    double Wk = 0.0;
                    for (int a = 0; a < o.nsel; ++a) {
                        const contrib_t *e = &cb[o.sel[a]];
                        const double *c = feats + (int64_t)e->id * C;
                        for (int ch = 0; ch < C; ++ch) f[ch] += e->w * c[ch];
                        Wk += e->w;
                    }
                    if (p->renorm && o.nsel > 0)
                        for (int ch = 0; ch < C; ++ch) f[ch] /= Wk;
                }
            }
            if (K > 0) {
                for (int a = 0; a < K; ++a) {
                    int has = a < o.nsel;
                    const contrib_t *e = has ? &cb[o.sel[a]] : NULL;
                    if (ids) ids[pix * K + a] = has ? e->id : -1;
                    if (wout) wout[pix * K + a] = has ? e->w : 0.0;
                    if (pos) pos[pix * K + a] = has ? e->pos : -1;
                }
            }
        }
        free(cb);
    }
    if (counters) { counters[0] = n_eval; counters[1] = n_contrib; }
    release(&sp);
}

/* ================================================================== */
/* 4. analytic gradients (chain rule of sections 1 and 3)               */
/* ================================================================== */

/* d t_u / d q_hat and d t_v / d q_hat for q_hat = (w, x, y, z) */
static void dframe(const double q[4], double dtu[4][3], double dtv[4][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double a[4][3] = {{0, 2 * z, -2 * y}, {0, 2 * y, 2 * z}, {-4 * y, 2 * x, -2 * w}, {-4 * z, 2 * w, 2 * x}};
    double b[4][3] = {{-2 * z, 0, 2 * x}, {2 * y, -4 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, -4 * z, 2 * y}};
    memcpy(dtu, a, sizeof a);
    memcpy(dtv, b, sizeof b);
}

/*
 * Gradients of L = sum_x [ gF(x).F(x) + grgb(x).RGB(x) + gT(x) T(x) ] for
 * the same view/order arguments as orc_render (gT may be NULL).  The
 * selection set, skips, stops, clamps and binning are held fixed.
 * Outputs (accumulated, caller zeroes): g_means[N*3], g_scales[N*2],
 * g_quats[N*4], g_opac[N], g_rgb[N*3], g_feat[N*C], and optionally the
 * per-surfel derivative w.r.t. the rows of T, g_T[N*9].  flip[H*W] (may
 * be NULL): the per-pixel borderline outcomes of orc_render, held fixed
 * like every other decision.
 * g_abs[N*10] (optional, accumulated): the same chain evaluated over
 * magnitudes, per surfel (means 3, scales 2, quats 4, opacity 1): every
 * sum and product of the chain, from the upstream gradients through
 * dL/dalpha, the ray-splat quotients, the cross products and the T-row
 * sums to the parameters, is taken over the absolute values of its
 * operands.  This is the scale of the rounding error of a finite-precision
 * evaluation of the same chain under cancellation (forward error
 * analysis), used for test tolerances; it is >= |gradient| entry by entry.
 */
void orc_render_backward(int64_t N, const double *means, const double *scales, const double *quats,
                         const double *opac, const double *rgb, const double *feats, const orc_cam *cam,
                         const orc_params *p, const int32_t *ranges, const int32_t *sorted_ids,
                         const int32_t *visible, const float *zkey,
                         const double *gF, const double *grgb, const double *gT,
                         double *g_means, double *g_scales, double *g_quats, double *g_opac,
                         double *g_rgb, double *g_feat, double *g_Tmat, double *g_abs,
                         const uint32_t *flip)
{
    const int W = cam->width, H = cam->height, ts = p->tile_size, C = p->C, K = p->K;
    const int tiles_x = (W + ts - 1) / ts;
    scene_prep sp;
    prepare(N, means, scales, quats, opac, cam, p, visible, zkey, ranges == NULL, &sp);
    double *dT = (double *)calloc((size_t)(N > 0 ? N : 1) * 9, sizeof(double));
    double *dTa = g_abs ? (double *)calloc((size_t)(N > 0 ? N : 1) * 9, sizeof(double)) : NULL;
    int64_t cap = ranges ? 0 : sp.n_order;
    if (ranges) {
        int nt = tiles_x * ((H + ts - 1) / ts);
        for (int t = 0; t < nt; ++t) {
            int64_t len = ranges[2 * t + 1] - ranges[2 * t];
            if (len > cap) cap = len;
        }
    }
    contrib_t *cb = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(cap > 0 ? cap : 1));
    double *s = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    double *sa = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    char *insel = (char *)malloc((size_t)(cap > 0 ? cap : 1));
    for (int py = 0; py < H; ++py) {
        for (int px = 0; px < W; ++px) {
            const int32_t *cand;
            int32_t n_cand;
            if (ranges) {
                int t = (py / ts) * tiles_x + px / ts;
                cand = sorted_ids + ranges[2 * t];
                n_cand = ranges[2 * t + 1] - ranges[2 * t];
            } else {
                cand = sp.order;
                n_cand = sp.n_order;
            }
            const double x = px + 0.5, y = py + 0.5;
            const int64_t pix = (int64_t)py * W + px;
            pix_out o;
            composite_pixel(sp.geo, opac, rgb, cam, p, cand, n_cand, x, y, flip ? flip[pix] : 0u, cb, &o);
            const double *gf = gF ? gF + pix * C : NULL;
            const double *gc = grgb + 3 * pix;
            const double gt = gT ? gT[pix] : 0.0;
            const int n = o.n_contrib;
            memset(insel, K == 0 ? 1 : 0, (size_t)(n > 0 ? n : 1));
            if (K > 0) for (int a = 0; a < o.nsel; ++a) insel[o.sel[a]] = 1;
            /* renormalised Top-K, F = sum_K w c / W: dL/dw_i = (c_i.gF - Fg) / W
             * with Fg = F.gF, and dL/dc_i = (w_i / W) gF */
            double Wk = 1.0, Fg = 0.0, Fga = 0.0;
            const int renorm = K > 0 && p->renorm && o.nsel > 0 && gf;
            if (renorm) {
                Wk = 0.0;
                for (int a = 0; a < o.nsel; ++a) Wk += cb[o.sel[a]].w;
                for (int a = 0; a < o.nsel; ++a) {
                    const contrib_t *e = &cb[o.sel[a]];
                    const double *c = feats + (int64_t)e->id * C;
                    double d = 0.0, da = 0.0;
                    for (int ch = 0; ch < C; ++ch) d += c[ch] * gf[ch];
                    for (int ch = 0; ch < C; ++ch) da += fabs(c[ch] * gf[ch]);
                    Fg += e->w / Wk * d;
                    Fga += e->w / Wk * da;
                }
            }
            /* s_i: what each blending weight multiplies */
            for (int i = 0; i < n; ++i) {
                const int id = cb[i].id;
                double v = 0.0, va = 0.0;
                for (int k = 0; k < 3; ++k) v += rgb[3 * id + k] * gc[k];
                for (int k = 0; k < 3; ++k) va += fabs(rgb[3 * id + k] * gc[k]);
                if (insel[i] && gf) {
                    const double *c = feats + (int64_t)id * C;
                    double d = 0.0, da = 0.0;
                    for (int ch = 0; ch < C; ++ch) d += c[ch] * gf[ch];
                    for (int ch = 0; ch < C; ++ch) da += fabs(c[ch] * gf[ch]);
                    v += renorm ? (d - Fg) / Wk : d;
                    va += renorm ? (da + Fga) / Wk : da;
                }
                s[i] = v;
                sa[i] = va;
                for (int k = 0; k < 3; ++k) g_rgb[3 * id + k] += cb[i].w * gc[k];
                if (insel[i] && gf)
                    for (int ch = 0; ch < C; ++ch) g_feat[(int64_t)id * C + ch] += cb[i].w / Wk * gf[ch];
            }
            /* dL/dalpha_j = T_j s_j - (sum_{i>j} w_i s_i + T_final (bg.grgb + gT)) / (1 - alpha_j) */
            double tail = o.T * (p->bg[0] * gc[0] + p->bg[1] * gc[1] + p->bg[2] * gc[2] + gt);
            double taila = o.T * (fabs(p->bg[0] * gc[0]) + fabs(p->bg[1] * gc[1]) + fabs(p->bg[2] * gc[2]) + fabs(gt));
            for (int j = n - 1; j >= 0; --j) {
                const contrib_t *e = &cb[j];
                const int id = e->id;
                double dal = e->T * s[j] - tail / (1.0 - e->alpha);
                const double dala = e->T * sa[j] + taila / (1.0 - e->alpha);
                tail += e->w * s[j];
                taila += e->w * sa[j];
                if (!(e->oG < p->alpha_max)) continue; /* clamped: flat */
                double G = e->oG / opac[id];
                g_opac[id] += dal * G;
                if (g_abs) g_abs[10 * (int64_t)id + 9] += dala * G;
                double drho = dal * (-0.5 * e->oG);
                if (e->scr) {
                    /* screen term: rho = 2 |x - c|^2 with c = (T1_2, T2_2) / Tw_2 */
                    const geo64 *gg = &sp.geo[id];
                    const double dcx = -4.0 * e->sx * drho, dcy = -4.0 * e->sy * drho, w2 = gg->T[2][2];
                    double *d = dT + 9 * (int64_t)id;
                    d[2] += dcx / w2;
                    d[5] += dcy / w2;
                    d[8] -= (dcx * gg->T[0][2] + dcy * gg->T[1][2]) / (w2 * w2);
                    if (dTa) {
                        const double ra = dala * 0.5 * e->oG, ax = 4.0 * fabs(e->sx) * ra, ay = 4.0 * fabs(e->sy) * ra;
                        double *da = dTa + 9 * (int64_t)id;
                        da[2] += ax / fabs(w2);
                        da[5] += ay / fabs(w2);
                        da[8] += (ax * fabs(gg->T[0][2]) + ay * fabs(gg->T[1][2])) / (w2 * w2);
                    }
                    continue;
                }
                double du = 2.0 * e->u * drho, dv = 2.0 * e->v * drho;
                double gcv[3] = {du / e->c[2], dv / e->c[2], -(du * e->u + dv * e->v) / e->c[2]};
                double dhx[3], dhy[3];
                cross3(e->hy, gcv, dhx);   /* d/dhx (hx x hy).g = hy x g */
                cross3(gcv, e->hx, dhy);   /* d/dhy (hx x hy).g = g x hx */
                double *d = dT + 9 * (int64_t)id;
                for (int k = 0; k < 3; ++k) {
                    d[k] += dhx[k];
                    d[3 + k] += dhy[k];
                    d[6 + k] += -x * dhx[k] - y * dhy[k];
                }
                if (dTa) { /* the same steps over magnitudes */
                    const double dra = dala * 0.5 * e->oG;
                    const double dua = 2.0 * fabs(e->u) * dra, dva = 2.0 * fabs(e->v) * dra;
                    const double ic = 1.0 / fabs(e->c[2]);
                    const double ga[3] = {dua * ic, dva * ic, (dua * fabs(e->u) + dva * fabs(e->v)) * ic};
                    const double ax[3] = {fabs(e->hx[0]), fabs(e->hx[1]), fabs(e->hx[2])};
                    const double ay[3] = {fabs(e->hy[0]), fabs(e->hy[1]), fabs(e->hy[2])};
                    const double ahx[3] = {ay[1] * ga[2] + ay[2] * ga[1], ay[2] * ga[0] + ay[0] * ga[2],
                                           ay[0] * ga[1] + ay[1] * ga[0]};
                    const double ahy[3] = {ga[1] * ax[2] + ga[2] * ax[1], ga[2] * ax[0] + ga[0] * ax[2],
                                           ga[0] * ax[1] + ga[1] * ax[0]};
                    double *da = dTa + 9 * (int64_t)id;
                    for (int k = 0; k < 3; ++k) {
                        da[k] += ahx[k];
                        da[3 + k] += ahy[k];
                        da[6 + k] += x * ahx[k] + y * ahy[k];
                    }
                }
            }
        }
    }
    /* T = Kcam [a_u | a_v | p_c] -> surfel parameters */
    for (int64_t i = 0; i < N; ++i) {
        const double *d = dT + 9 * i;
        if (g_Tmat) for (int k = 0; k < 9; ++k) g_Tmat[9 * i + k] += d[k];
        if (!sp.geo[i].ok) continue;
        double R[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) R[3 * r + c] = cam->viewmat[4 * r + c];
        double dcol[3][3]; /* dL/d(a_u), dL/d(a_v), dL/d(p_c) */
        for (int c = 0; c < 3; ++c) {
            dcol[c][0] = cam->fx * d[c];
            dcol[c][1] = cam->fy * d[3 + c];
            dcol[c][2] = cam->cx * d[c] + cam->cy * d[3 + c] + d[6 + c];
        }
        /* p_c = R p + t */
        for (int k = 0; k < 3; ++k)
            g_means[3 * i + k] += R[k] * dcol[2][0] + R[3 + k] * dcol[2][1] + R[6 + k] * dcol[2][2];
        double tu[3], tv[3], nn[3], Rtu[3], Rtv[3];
        frame64(quats + 4 * i, tu, tv, nn);
        matvec3(R, tu, Rtu);
        matvec3(R, tv, Rtv);
        g_scales[2 * i] += Rtu[0] * dcol[0][0] + Rtu[1] * dcol[0][1] + Rtu[2] * dcol[0][2];
        g_scales[2 * i + 1] += Rtv[0] * dcol[1][0] + Rtv[1] * dcol[1][1] + Rtv[2] * dcol[1][2];
        double dtu[3], dtv[3];
        for (int k = 0; k < 3; ++k) {
            dtu[k] = scales[2 * i] * (R[k] * dcol[0][0] + R[3 + k] * dcol[0][1] + R[6 + k] * dcol[0][2]);
            dtv[k] = scales[2 * i + 1] * (R[k] * dcol[1][0] + R[3 + k] * dcol[1][1] + R[6 + k] * dcol[1][2]);
        }
        const double *q = quats + 4 * i;
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qh[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
        double Ju[4][3], Jv[4][3], dqh[4];
        dframe(qh, Ju, Jv);
        for (int a = 0; a < 4; ++a)
            dqh[a] = Ju[a][0] * dtu[0] + Ju[a][1] * dtu[1] + Ju[a][2] * dtu[2] +
                     Jv[a][0] * dtv[0] + Jv[a][1] * dtv[1] + Jv[a][2] * dtv[2];
        double dot = dqh[0] * qh[0] + dqh[1] * qh[1] + dqh[2] * qh[2] + dqh[3] * qh[3];
        for (int a = 0; a < 4; ++a) g_quats[4 * i + a] += (dqh[a] - dot * qh[a]) / qn;
        if (dTa) { /* the same chain over magnitudes */
            const double *da = dTa + 9 * i;
            double acol[3][3], au[3], av[3], aqh[4], adot = 0.0;
            double *ga = g_abs + 10 * i;
            for (int c = 0; c < 3; ++c) {
                acol[c][0] = cam->fx * da[c];
                acol[c][1] = cam->fy * da[3 + c];
                acol[c][2] = fabs(cam->cx) * da[c] + fabs(cam->cy) * da[3 + c] + da[6 + c];
            }
            for (int k = 0; k < 3; ++k) {
                ga[k] += fabs(R[k]) * acol[2][0] + fabs(R[3 + k]) * acol[2][1] + fabs(R[6 + k]) * acol[2][2];
                au[k] = scales[2 * i] * (fabs(R[k]) * acol[0][0] + fabs(R[3 + k]) * acol[0][1] + fabs(R[6 + k]) * acol[0][2]);
                av[k] = scales[2 * i + 1] * (fabs(R[k]) * acol[1][0] + fabs(R[3 + k]) * acol[1][1] + fabs(R[6 + k]) * acol[1][2]);
            }
            ga[3] += fabs(Rtu[0]) * acol[0][0] + fabs(Rtu[1]) * acol[0][1] + fabs(Rtu[2]) * acol[0][2];
            ga[4] += fabs(Rtv[0]) * acol[1][0] + fabs(Rtv[1]) * acol[1][1] + fabs(Rtv[2]) * acol[1][2];
            for (int a = 0; a < 4; ++a) {
                aqh[a] = 0.0;
                for (int k = 0; k < 3; ++k) aqh[a] += fabs(Ju[a][k]) * au[k] + fabs(Jv[a][k]) * av[k];
                adot += aqh[a] * fabs(qh[a]);
            }
            for (int a = 0; a < 4; ++a) ga[5 + a] += (aqh[a] + adot * fabs(qh[a])) / qn;
        }
    }
    free(dT); free(dTa); free(cb); free(s); free(sa); free(insel);
    release(&sp);
}

/* ================================================================== */
/* 5. small helpers exported for closed-form checks                     */
/* ================================================================== */

/* FP64 T rows (T[9]), centre depth, cos(normal, view ray) and cull flag */
void orc_geometry(int64_t N, const double *means, const double *scales, const double *quats,
                  const double *opac, const orc_cam *cam, const orc_params *p,
                  double *T, double *z, double *cosang, int32_t *ok)
{
    for (int64_t i = 0; i < N; ++i) {
        geo64 g;
        geometry64(means + 3 * i, scales + 2 * i, quats + 4 * i, opac[i], cam, p, &g);
        if (T) for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) T[9 * i + 3 * r + c] = g.T[r][c];
        if (z) z[i] = g.z;
        if (cosang) cosang[i] = g.cosang;
        if (ok) ok[i] = g.ok;
    }
}

/* (u, v, z_hit, valid) of M pixel points for one T */
void orc_ray_splat(const double *T, int64_t M, const double *xy, double near, double *uvz, int32_t *valid)
{
    double Tm[3][3];
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) Tm[r][c] = T[3 * r + c];
    for (int64_t k = 0; k < M; ++k) {
        double u = 0, v = 0, zh = 0, hx[3], hy[3], c[3];
        valid[k] = ray_splat64(Tm, xy[2 * k], xy[2 * k + 1], near, &u, &v, &zh, hx, hy, c);
        uvz[3 * k] = u; uvz[3 * k + 1] = v; uvz[3 * k + 2] = zh;
    }
}

/*
 * Conservativeness of a binning: for each surfel that passes the cull rules
 * of the mirror, every pixel whose FP64 alpha reaches alpha_min must lie in
 * one of the surfel's tiles.  Returns the number of violating (pixel, surfel)
 * pairs; *n_checked = number of (pixel, surfel) pairs with alpha >= alpha_min.
 */
int64_t orc_check_conservative(int64_t N, const float *means, const float *scales, const float *quats,
                               const float *opac, const orc_cam *cam, const orc_params *p, int mode,
                               int64_t *n_checked)
{
    const int W = cam->width, H = cam->height, ts = p->tile_size;
    const int tiles_x = (W + ts - 1) / ts, tiles_y = (H + ts - 1) / ts;
    int64_t bad = 0, checked = 0;
    char *mark = (char *)malloc((size_t)tiles_x * tiles_y);
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)tiles_x * tiles_y);
    for (int64_t i = 0; i < N; ++i) {
        mirror_rec r;
        mirror_project(means + 3 * i, scales + 2 * i, quats + 4 * i, opac[i], cam, p, mode, &r);
        if (r.culled_by_rule) continue;
        memset(mark, 0, (size_t)tiles_x * tiles_y);
        int64_t n = tiles_of(&r, cam, p, mode, buf, (int64_t)tiles_x * tiles_y);
        for (int64_t k = 0; k < n; ++k) mark[buf[k]] = 1;
        geo64 g;
        double dm[3], ds[2], dq[4];
        for (int k = 0; k < 3; ++k) dm[k] = means[3 * i + k];
        for (int k = 0; k < 2; ++k) ds[k] = scales[2 * i + k];
        for (int k = 0; k < 4; ++k) dq[k] = quats[4 * i + k];
        geometry64(dm, ds, dq, opac[i], cam, p, &g);
        /* FP64 search window: the ellipse of twice the cutoff (whole image
         * when that conic is not an ellipse) */
        int x0 = 0, x1 = W - 1, y0 = 0, y1 = H - 1;
        {
            double a[3][3], m[3][3], q[6];
            for (int r0 = 0; r0 < 3; ++r0) for (int c0 = 0; c0 < 3; ++c0) a[r0][c0] = g.T[r0][c0];
            double c0v[3] = {a[0][0], a[1][0], a[2][0]}, c1v[3] = {a[0][1], a[1][1], a[2][1]},
                   c2v[3] = {a[0][2], a[1][2], a[2][2]};
            cross3(c1v, c2v, m[0]); cross3(c2v, c0v, m[1]); cross3(c0v, c1v, m[2]);
            double kk = 2.0 * 2.0 * log(opac[i] / (double)p->alpha_min) + 1.0;
            const int ia[6] = {0, 0, 1, 0, 1, 2}, ib[6] = {0, 1, 1, 2, 2, 2};
            for (int k = 0; k < 6; ++k)
                q[k] = m[0][ia[k]] * m[0][ib[k]] + m[1][ia[k]] * m[1][ib[k]] - kk * m[2][ia[k]] * m[2][ib[k]];
            double gg = q[0] * q[2] - q[1] * q[1];
            if (q[0] > 0 && gg > 0) {
                double X0 = (q[1] * q[4] - q[2] * q[3]) / gg, Y0 = (q[1] * q[3] - q[0] * q[4]) / gg;
                double Fp = q[5] + q[3] * X0 + q[4] * Y0;
                double lx = 1e30, hxp = -1e30, ly = 1e30, hyp = -1e30;
                if (Fp < 0) {
                    double hxx = sqrt(-Fp * q[2] / gg) + 2.0, hyy = sqrt(-Fp * q[0] / gg) + 2.0;
                    lx = floor(X0 - hxx); hxp = ceil(X0 + hxx); ly = floor(Y0 - hyy); hyp = ceil(Y0 + hyy);
                }
                if (p->lowpass) { /* the screen disc 2 |x - c|^2 <= k^2, widened */
                    double rr = sqrt(log(opac[i] / (double)p->alpha_min)) + 2.0;
                    lx = fmin(lx, floor(g.cxp - rr)); hxp = fmax(hxp, ceil(g.cxp + rr));
                    ly = fmin(ly, floor(g.cyp - rr)); hyp = fmax(hyp, ceil(g.cyp + rr));
                }
                if (lx > hxp) continue;
                if (hxp < 0 || lx > W - 1 || hyp < 0 || ly > H - 1) continue;
                x0 = lx < 0 ? 0 : (int)lx; x1 = hxp > W - 1 ? W - 1 : (int)hxp;
                y0 = ly < 0 ? 0 : (int)ly; y1 = hyp > H - 1 ? H - 1 : (int)hyp;
            }
        }
        for (int py = y0; py <= y1; ++py)
            for (int px = x0; px <= x1; ++px) {
                double u = 0.0, v = 0.0, zh = 0.0, hx[3], hy[3], c[3];
                const int obj = ray_splat64(g.T, px + 0.5, py + 0.5, -INFINITY, &u, &v, &zh, hx, hy, c);
                double rho = obj ? u * u + v * v : INFINITY;
                if (p->lowpass) {
                    const double sx = px + 0.5 - g.cxp, sy = py + 0.5 - g.cyp, rs = 2.0 * (sx * sx + sy * sy);
                    if (!(rho <= rs)) { rho = rs; zh = g.z; }
                } else if (!obj) {
                    continue;
                }
                if (!(zh > cam->near_plane)) continue;
                double a = opac[i] * exp(-0.5 * rho);
                if (a < p->alpha_min) continue;
                ++checked;
                if (!mark[(py / ts) * tiles_x + px / ts]) ++bad;
            }
    }
    free(mark); free(buf);
    if (n_checked) *n_checked = checked;
    return bad;
}

/* ================================================================== */
/* 6. query-guided instance labels (Sec. 3.3)                           */
/* ================================================================== */

/*
 * Instance label distribution of every scene Gaussian g over the nq
 * instance queries, following the paper's steps in order:
 *   S(q, g) = sigmoid(f_q . f_ins(g))                 (feature similarity)
 *   D(q, g) = phi_q(p_g) / phi_q(p_q)                 (spatial proximity)
 *           = exp(-1/2 (p_g - p_q)^T Sigma_q^-1 (p_g - p_q)),
 *     phi_q the density of the query's Gaussian N(p_q, Sigma_q); the
 *     normalising constant cancels in the ratio;
 *   A(q, g) = S(q, g) D(q, g)                         (attention)
 *   l_ins(g) = softmax over q of A(q, g).
 * Scene Gaussians enter as points (their centres), as the paper states.
 * Inputs: f_ins [N, dim], means [N, 3], f_q [nq, dim], p_q [nq, 3],
 * prec [nq, 6] = Sigma_q^-1 entries (xx, yy, zz, xy, xz, yz).
 * Output: labels [N, nq].
 */
void orc_query_labels(int64_t N, int32_t nq, int32_t dim, const double *f_ins, const double *means,
                      const double *f_q, const double *p_q, const double *prec, double *labels)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < N; ++g) {
        double *l = labels + g * nq;
        double sum = 0.0;
        for (int q = 0; q < nq; ++q) {
            double dot = 0.0;
            for (int k = 0; k < dim; ++k) dot += f_q[(int64_t)q * dim + k] * f_ins[g * dim + k];
            const double S = 1.0 / (1.0 + exp(-dot));
            const double d[3] = {means[3 * g] - p_q[3 * q], means[3 * g + 1] - p_q[3 * q + 1],
                                 means[3 * g + 2] - p_q[3 * q + 2]};
            const double *P = prec + 6 * (int64_t)q;
            const double Pm[3][3] = {{P[0], P[3], P[4]}, {P[3], P[1], P[5]}, {P[4], P[5], P[2]}};
            double quad = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) quad += d[a] * Pm[a][b] * d[b];
            const double D = exp(-0.5 * quad);
            const double A = S * D;
            l[q] = exp(A);
            sum += l[q];
        }
        for (int q = 0; q < nq; ++q) l[q] /= sum;
    }
}

/* ================================================================== */
/* 7. view-dependent colour: real spherical harmonics (Sec. 3.1)        */
/* ================================================================== */

/*
 * The surfel colour c_i is view dependent (Sec. 3.1).  Reading: as in the
 * 2DGS/3DGS base models, real spherical harmonics of degree <= 3 of the
 * unit direction d from the camera centre to the surfel centre, plus 1/2,
 * clamped at 0 per channel:  c = max(0, sum_b k_b Y_b(d) + 1/2).
 * Basis index b = l^2 + l + m.  Real harmonics without the Condon-Shortley
 * sign, written in Cartesian form on the unit sphere from the textbook
 * definition: with A_m + i B_m = (x + i y)^m and L_l^m = d^m P_l / dz^m
 * (P_l the Legendre polynomial),
 *   Y_l0  = n_l0 P_l(z),
 *   Y_lm  = sqrt(2) n_lm L_l^m(z) A_m(x, y),   m > 0,
 *   Y_l-m = sqrt(2) n_lm L_l^m(z) B_m(x, y),   m > 0,
 * n_lm = sqrt((2l + 1) / (4 pi) (l - m)! / (l + m)!).
 * grad[b][3] (optional) = the partial derivatives of that polynomial in
 * (x, y, z), for the chain rule through the direction.
 */
static void legendre_poly(int l, double c[4])  /* coefficients of P_l, ascending powers */
{
    double p0[4] = {1, 0, 0, 0}, p1[4] = {0, 1, 0, 0};
    if (l == 0) { memcpy(c, p0, sizeof p0); return; }
    for (int k = 1; k < l; ++k) { /* (k+1) P_{k+1} = (2k+1) z P_k - k P_{k-1} */
        double p2[4] = {0, 0, 0, 0};
        for (int j = 0; j < 3; ++j) p2[j + 1] += (2 * k + 1) * p1[j];
        for (int j = 0; j < 4; ++j) p2[j] = (p2[j] - k * p0[j]) / (k + 1);
        memcpy(p0, p1, sizeof p1);
        memcpy(p1, p2, sizeof p2);
    }
    memcpy(c, p1, sizeof p1);
}

static double poly_deriv_eval(const double c[4], int m, double z)  /* d^m/dz^m of the polynomial at z */
{
    double d[4];
    memcpy(d, c, sizeof d);
    for (int k = 0; k < m; ++k) {
        for (int j = 0; j < 3; ++j) d[j] = (j + 1) * d[j + 1];
        d[3] = 0.0;
    }
    return ((d[3] * z + d[2]) * z + d[1]) * z + d[0];
}

static double factorial(int n) { double f = 1.0; for (int k = 2; k <= n; ++k) f *= k; return f; }

void orc_sh_basis(int deg, const double dir[3], double *Y, double *grad)
{
    const double x = dir[0], y = dir[1], z = dir[2];
    double A[5], B[5]; /* (x + i y)^m */
    A[0] = 1.0; B[0] = 0.0;
    for (int m = 1; m <= 4; ++m) { A[m] = x * A[m - 1] - y * B[m - 1]; B[m] = x * B[m - 1] + y * A[m - 1]; }
    for (int l = 0; l <= deg; ++l) {
        double P[4];
        legendre_poly(l, P);
        for (int m = -l; m <= l; ++m) {
            const int am = m < 0 ? -m : m, b = l * l + l + m;
            const double n = sqrt((2 * l + 1) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am)) *
                             (am ? sqrt(2.0) : 1.0);
            const double L = poly_deriv_eval(P, am, z), Lz = poly_deriv_eval(P, am + 1, z);
            const double T = m > 0 ? A[am] : (m < 0 ? B[am] : 1.0);
            /* d A_m / dx = m A_{m-1}, d A_m / dy = -m B_{m-1}; d B_m / dx = m B_{m-1}, d B_m / dy = m A_{m-1} */
            double Tx = 0.0, Ty = 0.0;
            if (m > 0) { Tx = am * A[am - 1]; Ty = -am * B[am - 1]; }
            if (m < 0) { Tx = am * B[am - 1]; Ty = am * A[am - 1]; }
            Y[b] = n * L * T;
            if (grad) { grad[3 * b] = n * L * Tx; grad[3 * b + 1] = n * L * Ty; grad[3 * b + 2] = n * Lz * T; }
        }
    }
}

/* camera centre of a world-to-camera [R | t]: -R^T t */
static void cam_centre(const orc_cam *cam, double C[3])
{
    for (int k = 0; k < 3; ++k)
        C[k] = -(cam->viewmat[k] * cam->viewmat[3] + cam->viewmat[4 + k] * cam->viewmat[7] +
                 cam->viewmat[8 + k] * cam->viewmat[11]);
}

/*
 * Per-surfel colours for one camera: rgb[N, 3] = max(0, sum_b coef[N, B, 3]
 * Y_b(d) + 1/2), d = (p - C) / |p - C|, B = (deg + 1)^2.
 */
void orc_sh_colors(int64_t N, int deg, const double *coef, const double *means, const orc_cam *cam, double *rgb)
{
    const int nb = (deg + 1) * (deg + 1);
    double C[3];
    cam_centre(cam, C);
    for (int64_t i = 0; i < N; ++i) {
        double v[3] = {means[3 * i] - C[0], means[3 * i + 1] - C[1], means[3 * i + 2] - C[2]};
        const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double d[3] = {v[0] / r, v[1] / r, v[2] / r};
        double Y[16];
        orc_sh_basis(deg, d, Y, NULL);
        for (int ch = 0; ch < 3; ++ch) {
            double c = 0.5;
            for (int b = 0; b < nb; ++b) c += coef[(i * nb + b) * 3 + ch] * Y[b];
            rgb[3 * i + ch] = c > 0.0 ? c : 0.0;
        }
    }
}

/*
 * Chain rule of orc_sh_colors for upstream colour gradients g_rgb[N, 3] of
 * one camera: adds dL/dcoef to g_coef[N, B, 3] and the direction term to
 * g_means[N, 3] (d = v / |v| gives dd/dv = (I - d d^T) / |v|); a clamped
 * channel passes nothing.  g_abs (optional, [N, 10] as in the render
 * backward) gets the magnitude of the direction term's chain in its means
 * columns.
 */
void orc_sh_backward(int64_t N, int deg, const double *coef, const double *means, const orc_cam *cam,
                     const double *g_rgb, double *g_coef, double *g_means, double *g_abs)
{
    const int nb = (deg + 1) * (deg + 1);
    double C[3];
    cam_centre(cam, C);
    for (int64_t i = 0; i < N; ++i) {
        double v[3] = {means[3 * i] - C[0], means[3 * i + 1] - C[1], means[3 * i + 2] - C[2]};
        const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double d[3] = {v[0] / r, v[1] / r, v[2] / r};
        double Y[16], G[48];
        orc_sh_basis(deg, d, Y, G);
        double gd[3] = {0, 0, 0}, gda[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            double c = 0.5;
            for (int b = 0; b < nb; ++b) c += coef[(i * nb + b) * 3 + ch] * Y[b];
            if (!(c > 0.0)) continue;
            const double g = g_rgb[3 * i + ch];
            for (int b = 0; b < nb; ++b) {
                g_coef[(i * nb + b) * 3 + ch] += Y[b] * g;
                for (int k = 0; k < 3; ++k) {
                    gd[k] += g * coef[(i * nb + b) * 3 + ch] * G[3 * b + k];
                    gda[k] += fabs(g * coef[(i * nb + b) * 3 + ch] * G[3 * b + k]);
                }
            }
        }
        const double dot = d[0] * gd[0] + d[1] * gd[1] + d[2] * gd[2];
        const double dota = fabs(d[0]) * gda[0] + fabs(d[1]) * gda[1] + fabs(d[2]) * gda[2];
        for (int k = 0; k < 3; ++k) {
            g_means[3 * i + k] += (gd[k] - d[k] * dot) / r;
            if (g_abs) g_abs[10 * i + k] += (gda[k] + fabs(d[k]) * dota) / r;
        }
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
