/*
 * rg_oracle.c -- plain, slow CPU oracle of the RoofGS forward render.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library. The GPU renderer
 * never links, includes or calls it, and it shares no code with the renderer.
 *
 * What it computes (paper: "RoofGS: Roofline-Guided End-to-End Acceleration of
 * 3D Gaussian Splatting"):
 *   - the per-pixel front-to-back alpha blend of Sec. III-D, Eq. (7)
 *     alpha_computation, with the power of Eq. (10), the opacity of
 *     Eqs. (11)-(12) (clamp at 0.99), in FP64;
 *   - in RoofGS mode the folded exponent P = p + log o of Eq. (17)/(21), the
 *     skip of every pair outside the range of Eq. (23) [-ln 255, 0], and
 *     optionally the bit-level exponential of Eq. (24);
 *   - the tile binning and sort key in FP32 with a pinned operation order
 *     (RoofGS mode: the box and per-tile-row extent of the alpha = 1/255
 *     ellipse, reading of the Speedy-Splat culling adopted in Sec. IV-A.3):
 *     the 64-bit tile|float-depth key of Sec. IV-A.2 (baseline) and the
 *     resolution-adaptive 32-bit tile|quantized-depth key of Eq. (9)
 *     depth_quant with b_t = ceil(log2(TxTy)), b_d = 32 - b_t.
 *
 * Readings of what the paper leaves to 3DGS (projection, EWA covariance,
 * spherical harmonics) are the plain definitions: world->camera p = R mu + t,
 * Sigma = Q diag(s)^2 Q^T for the unit quaternion's rotation Q, the EWA
 * covariance J W Sigma W^T J^T + 0.3 I with the perspective Jacobian J
 * (tangent clamped at 1.3x the half field of view), the pixel-centre
 * convention (pixel (i,j) sampled at (i,j)), real orthonormal spherical
 * harmonics up to degree 3 with colour = sum Y_k SH_k + 0.5 clamped to [0,1].
 *
 * The FP32 path uses only +, -, *, /, sqrt, floor, ceil, min and max, each a
 * single correctly rounded IEEE operation (this file must be compiled with
 * -ffp-contract=off). The GPU renderer implements the same operation order
 * independently, so culling, tile rectangles and keys are bit-exact.
 */
#include <complex.h>
#undef I /* the imaginary unit is written _Complex_I; I names integers below */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXACT 0
#define ORC_ROOFGS 1

#define ORC_EXP_EXACT 0  /* exp() in FP64 */
#define ORC_EXP_FAST64 1 /* Eq. (24) evaluated in real (FP64) arithmetic */
#define ORC_EXP_FAST32 2 /* Eq. (24) evaluated as one FP32 fma + truncation */

/* ln(255): the opacity threshold 1/255 in log space, Eq. (23). */
#define ORC_LN255 5.541263545158426
#define ORC_LN255F 5.541263545158426f
/* Schraudolph calibration constant of Eq. (24). */
#define ORC_SIGMA 0.045677

typedef struct {
    float R[9];  /* world -> camera rotation, row-major */
    float t[3];  /* world -> camera translation */
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear, zfar;
    float bg[3];
} orc_camera;

typedef struct {
    int32_t tile_w, tile_h, tiles_x, tiles_y;
    int32_t b_t, b_d;
    uint32_t qmax;
    float depth_scale;
} orc_layout;

/* Result of the FP32 binning path for one Gaussian. */
typedef struct {
    int32_t vis; /* 1 if it emits at least one tile entry */
    int32_t tx0, ty0, tx1, ty1;
    uint32_t qd;   /* RoofGS quantized depth, Eq. (9) */
    float z;       /* camera-space depth (FP32) */
    float u, v;    /* projected mean (FP32) */
    float rx, ry;  /* box half-extent in pixels (FP32) */
    /* RoofGS per-row test: level t, Sigma'_yy, and the row-extent constants */
    float tt, isc, ys, cc, kk;
    float xl, xh, yl, yh; /* pixel-centre box */
} orc_bin;

/* Per-Gaussian FP64 quantities for blending. */
typedef struct {
    double u, v, z;
    double a, b, c;           /* paper's (a, b, c): q = a dx^2 + b dx dy + c dy^2 */
    double s00, s01, s11;     /* EWA covariance Sigma' incl. 0.3 I */
    double gg;                /* exact mode: product of the natural row sizes of U (see below) */
    double op;                /* opacity o (exact) or log o (RoofGS) */
    double rgb[3];
} orc_g64;

/* ------------------------------------------------------------------------- */
/* Tile layout and the resolution-adaptive bit split (Sec. IV-A.2).            */
/* ------------------------------------------------------------------------- */

int orc_layout_compute(const orc_camera* c, int32_t tile_w, int32_t tile_h, orc_layout* L)
{
    if (tile_w <= 0 || tile_h <= 0 || c->width <= 0 || c->height <= 0) return -1;
    L->tile_w = tile_w;
    L->tile_h = tile_h;
    L->tiles_x = (c->width + tile_w - 1) / tile_w;
    L->tiles_y = (c->height + tile_h - 1) / tile_h;
    int64_t nt = (int64_t)L->tiles_x * (int64_t)L->tiles_y;
    int b = 0;
    while (((int64_t)1 << b) < nt) b++; /* b_t = ceil(log2 N_t) */
    if (b > 32) return -1;
    L->b_t = b;
    L->b_d = 32 - b; /* b_d = 32 - b_t */
    L->qmax = (L->b_d >= 32) ? 0xFFFFFFFFu : (uint32_t)((1ull << L->b_d) - 1ull);
    /* (2^b_d - 1) / (z_far - z_near), computed once in FP64, stored as FP32 */
    L->depth_scale = (float)((double)L->qmax / ((double)c->zfar - (double)c->znear));
    return 0;
}

/* ------------------------------------------------------------------------- */
/* FP32 pinned-order binning path.                                             */
/* ------------------------------------------------------------------------- */

static float fminf_(float a, float b) { return a < b ? a : b; }
static float fmaxf_(float a, float b) { return a > b ? a : b; }

/*
 * Culling, projected mean, box and tile rectangle of one Gaussian in FP32.
 * mode ORC_EXACT: 3-sigma box of the largest eigenvalue (plain 3DGS);
 * mode ORC_ROOFGS: opacity culling o < 1/255 and the exact axis-aligned box of
 * the alpha = 1/255 ellipse (reading of the Speedy-Splat culling, Sec. IV-A.3).
 * `op` is the opacity o in exact mode and log o in RoofGS mode.
 */
static void bin32(const float* m, const float* qin, const float* s, float op, int mode,
                  const orc_camera* c, const orc_layout* L, orc_bin* b)
{
    memset(b, 0, sizeof(*b));
    const float* R = c->R;
    float px = ((R[0] * m[0] + R[1] * m[1]) + R[2] * m[2]) + c->t[0];
    float py = ((R[3] * m[0] + R[4] * m[1]) + R[5] * m[2]) + c->t[1];
    float pz = ((R[6] * m[0] + R[7] * m[1]) + R[8] * m[2]) + c->t[2];
    b->z = pz;
    if (!(pz > c->znear) || !(pz <= c->zfar)) return; /* depth interval, Sec. IV-A.2 */
    if (mode == ORC_ROOFGS && !(op >= -ORC_LN255F)) return;

    float n2 = ((qin[0] * qin[0] + qin[1] * qin[1]) + qin[2] * qin[2]) + qin[3] * qin[3];
    if (!(n2 > 0.0f)) return;
    float rn = sqrtf(n2);
    float w = qin[0] / rn, x = qin[1] / rn, y = qin[2] / rn, z = qin[3] / rn;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float Q[9];
    Q[0] = 1.0f - 2.0f * (yy + zz); Q[1] = 2.0f * (xy - wz);        Q[2] = 2.0f * (xz + wy);
    Q[3] = 2.0f * (xy + wz);        Q[4] = 1.0f - 2.0f * (xx + zz); Q[5] = 2.0f * (yz - wx);
    Q[6] = 2.0f * (xz - wy);        Q[7] = 2.0f * (yz + wx);        Q[8] = 1.0f - 2.0f * (xx + yy);
    float M[9]; /* M = Q diag(s) */
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) M[3 * i + k] = Q[3 * i + k] * s[k];

    float xzr = px / pz, yzr = py / pz;
    float limx = 1.3f * ((0.5f * (float)c->width) / c->fx);
    float limy = 1.3f * ((0.5f * (float)c->height) / c->fy);
    float cxz = fminf_(limx, fmaxf_(-limx, xzr));
    float cyz = fminf_(limy, fmaxf_(-limy, yzr));
    float j00 = c->fx / pz, j11 = c->fy / pz;
    float j02 = -(j00 * cxz), j12 = -(j11 * cyz);
    float A[6]; /* A = J W, W = camera rotation */
    for (int k = 0; k < 3; k++) {
        A[k] = j00 * R[k] + j02 * R[6 + k];
        A[3 + k] = j11 * R[3 + k] + j12 * R[6 + k];
    }
    float U[6]; /* U = A M, Sigma' - 0.3 I = U U^T */
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            U[3 * i + k] = (A[3 * i] * M[k] + A[3 * i + 1] * M[3 + k]) + A[3 * i + 2] * M[6 + k];
    float sa = ((U[0] * U[0] + U[1] * U[1]) + U[2] * U[2]) + 0.3f;
    float sc = ((U[3] * U[3] + U[4] * U[4]) + U[5] * U[5]) + 0.3f;
    float sb = (U[0] * U[3] + U[1] * U[4]) + U[2] * U[5];

    float u = c->fx * xzr + c->cx;
    float v = c->fy * yzr + c->cy;
    float rx, ry;
    if (mode == ORC_EXACT) {
        float h = 0.5f * (sa - sc);
        float disc = sqrtf(h * h + sb * sb);
        float lmax = 0.5f * (sa + sc) + disc;
        float r = ceilf(3.0f * sqrtf(lmax));
        rx = r;
        ry = r;
    } else {
        float tt = 2.0f * (op + ORC_LN255F);
        rx = sqrtf(tt * sa);
        ry = sqrtf(tt * sc);
    }
    b->u = u; b->v = v; b->rx = rx; b->ry = ry;
    if (!isfinite(u) || !isfinite(v) || !isfinite(rx) || !isfinite(ry)) return;
    float xl = fmaxf_(ceilf(u - rx), 0.0f);
    float xh = fminf_(floorf(u + rx), (float)(c->width - 1));
    float yl = fmaxf_(ceilf(v - ry), 0.0f);
    float yh = fminf_(floorf(v + ry), (float)(c->height - 1));
    if (xl > xh || yl > yh) return;
    b->xl = xl; b->xh = xh; b->yl = yl; b->yh = yh;
    if (mode == ORC_ROOFGS) {
        /* Constants of the ellipse {d : d^T Sigma'^-1 d <= t}: for a band of
         * rows its x-extent is u + c dy +- k sqrt(t - dy^2 / Sigma'_yy) with
         * c = Sigma'_xy / Sigma'_yy, k = sqrt(det / Sigma'_yy), the right-most
         * point at dy = Sigma'_xy sqrt(t / Sigma'_xx); det by the Lagrange
         * identity det = |U0 x U1|^2 + 0.3 (|U0|^2 + |U1|^2) + 0.09. */
        float n0 = ((U[0] * U[0] + U[1] * U[1]) + U[2] * U[2]);
        float n1 = ((U[3] * U[3] + U[4] * U[4]) + U[5] * U[5]);
        float c0 = U[1] * U[5] - U[2] * U[4];
        float c1 = U[2] * U[3] - U[0] * U[5];
        float c2 = U[0] * U[4] - U[1] * U[3];
        float det = (((c0 * c0 + c1 * c1) + c2 * c2) + 0.3f * (n0 + n1)) + 0.09f;
        float tt = 2.0f * (op + ORC_LN255F);
        b->tt = tt;
        b->isc = 1.0f / sc;
        b->ys = sb * sqrtf(tt / sa);
        b->cc = sb / sc;
        b->kk = sqrtf(det / sc);
    }
    b->tx0 = (int32_t)xl / L->tile_w;
    b->tx1 = (int32_t)xh / L->tile_w;
    b->ty0 = (int32_t)yl / L->tile_h;
    b->ty1 = (int32_t)yh / L->tile_h;
    b->vis = 1;
    if (mode == ORC_ROOFGS) { /* Eq. (9) */
        float dq = (pz - c->znear) * L->depth_scale;
        dq = fmaxf_(dq, 0.0f);
        float fq = floorf(dq);
        float fqmax = (float)L->qmax;
        b->qd = (fq >= fqmax) ? L->qmax : (uint32_t)fq;
    }
}

static uint32_t f32_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Sort key of one (tile, Gaussian) entry. */
static uint64_t entry_key(const orc_bin* b, int mode, const orc_layout* L, int32_t tile)
{
    if (mode == ORC_EXACT) return ((uint64_t)(uint32_t)tile << 32) | (uint64_t)f32_bits(b->z);
    if (L->b_d >= 32) return (uint64_t)b->qd;
    return ((uint64_t)(uint32_t)tile << L->b_d) | (uint64_t)b->qd;
}

/*
 * RoofGS tile range of one tile row ty (reading of the Speedy-Splat culling of
 * Sec. IV-A.3): the x-extent of the alpha = 1/255 ellipse over the row's band
 * of pixel centres, clipped to the box; returns 0 if the row has no pixel
 * centre in it. Exact mode uses the whole rectangle row.
 */
static int row_range(const orc_bin* b, int mode, const orc_layout* L, int ty, int32_t* txa, int32_t* txb)
{
    if (mode == ORC_EXACT) {
        *txa = b->tx0;
        *txb = b->tx1;
        return 1;
    }
    float ya = fmaxf_((float)(ty * L->tile_h), b->yl);
    float yb = fminf_((float)(ty * L->tile_h + L->tile_h - 1), b->yh);
    float d0 = ya - b->v, d1 = yb - b->v;
    float dmax = fminf_(fmaxf_(b->ys, d0), d1);
    float dmin = fminf_(fmaxf_(-b->ys, d0), d1);
    float wr = sqrtf(fmaxf_(b->tt - (dmax * dmax) * b->isc, 0.0f));
    float wl = sqrtf(fmaxf_(b->tt - (dmin * dmin) * b->isc, 0.0f));
    float xr = (b->u + b->cc * dmax) + b->kk * wr;
    float xf = (b->u + b->cc * dmin) - b->kk * wl;
    float a0 = fmaxf_(ceilf(xf), b->xl);
    float a1 = fminf_(floorf(xr), b->xh);
    if (!(a0 <= a1)) return 0;
    *txa = (int32_t)a0 / L->tile_w;
    *txb = (int32_t)a1 / L->tile_w;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* FP64 definitions.                                                           */
/* ------------------------------------------------------------------------- */

/*
 * Real orthonormal spherical harmonics up to degree 3 at the unit direction
 * (x, y, z), index k = l^2 + l + m. Written from the closed forms
 * Y_lm = N_lm * (polynomial); the sign convention has no Condon-Shortley phase,
 * so Y_{1,-1}, Y_{1,0}, Y_{1,1} are positive multiples of y, z, x.
 */
void orc_sh_basis(double x, double y, double z, double* Y)
{
    const double pi = 3.14159265358979323846;
    Y[0] = 0.5 * sqrt(1.0 / pi);
    double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = k1 * y;
    Y[2] = k1 * z;
    Y[3] = k1 * x;
    double k2a = 0.5 * sqrt(15.0 / pi);
    double k20 = 0.25 * sqrt(5.0 / pi);
    double k22 = 0.25 * sqrt(15.0 / pi);
    Y[4] = k2a * x * y;
    Y[5] = k2a * y * z;
    Y[6] = k20 * (3.0 * z * z - 1.0);
    Y[7] = k2a * x * z;
    Y[8] = k22 * (x * x - y * y);
    double k33 = 0.25 * sqrt(35.0 / (2.0 * pi));
    double k32 = 0.5 * sqrt(105.0 / pi);
    double k31 = 0.25 * sqrt(21.0 / (2.0 * pi));
    double k30 = 0.25 * sqrt(7.0 / pi);
    double k32b = 0.25 * sqrt(105.0 / pi);
    Y[9] = k33 * y * (3.0 * x * x - y * y);
    Y[10] = k32 * x * y * z;
    Y[11] = k31 * y * (5.0 * z * z - 1.0);
    Y[12] = k30 * z * (5.0 * z * z - 3.0);
    Y[13] = k31 * x * (5.0 * z * z - 1.0);
    Y[14] = k32b * z * (x * x - y * y);
    Y[15] = k33 * x * (x * x - 3.0 * y * y);
}

/* Rotation matrix of the normalised quaternion (w, x, y, z), row-major. */
void orc_quat_to_rot(const double* qin, double* Q)
{
    double n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
    Q[0] = 1 - 2 * (y * y + z * z); Q[1] = 2 * (x * y - w * z);     Q[2] = 2 * (x * z + w * y);
    Q[3] = 2 * (x * y + w * z);     Q[4] = 1 - 2 * (x * x + z * z); Q[5] = 2 * (y * z - w * x);
    Q[6] = 2 * (x * z - w * y);     Q[7] = 2 * (y * z + w * x);     Q[8] = 1 - 2 * (x * x + y * y);
}

/* 3D covariance Sigma = Q diag(s)^2 Q^T (row-major 3x3). */
void orc_cov3d(const double* q, const double* s, double* S)
{
    double Q[9];
    orc_quat_to_rot(q, Q);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += Q[3 * i + k] * s[k] * s[k] * Q[3 * j + k];
            S[3 * i + j] = acc;
        }
}

/*
 * EWA projection of one Gaussian in FP64: camera-space mean, 2D mean (u, v),
 * Sigma' = J W Sigma W^T J^T + 0.3 I and its inverse in the paper's (a, b, c)
 * notation of Eq. (10): a = inv[0][0], b = 2 inv[0][1], c = inv[1][1].
 * out[0..9] = u, v, z, s00, s01, s11, a, b, c, det.
 */
void orc_project64(const float* mf, const float* qf, const float* sf, const orc_camera* c, double* out)
{
    double R[9], t[3], m[3], q[4], s[3];
    for (int i = 0; i < 9; i++) R[i] = c->R[i];
    for (int i = 0; i < 3; i++) { t[i] = c->t[i]; m[i] = mf[i]; s[i] = sf[i]; }
    for (int i = 0; i < 4; i++) q[i] = qf[i];
    double p[3];
    for (int i = 0; i < 3; i++) p[i] = R[3 * i] * m[0] + R[3 * i + 1] * m[1] + R[3 * i + 2] * m[2] + t[i];
    double S[9];
    orc_cov3d(q, s, S);
    double fx = c->fx, fy = c->fy;
    double limx = 1.3 * (0.5 * c->width / fx), limy = 1.3 * (0.5 * c->height / fy);
    double xz = p[0] / p[2], yz = p[1] / p[2];
    double cxz = xz < -limx ? -limx : (xz > limx ? limx : xz);
    double cyz = yz < -limy ? -limy : (yz > limy ? limy : yz);
    double J[6] = {fx / p[2], 0, -fx * cxz / p[2], 0, fy / p[2], -fy * cyz / p[2]};
    double T[6]; /* T = J R */
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            T[3 * i + k] = J[3 * i] * R[k] + J[3 * i + 1] * R[3 + k] + J[3 * i + 2] * R[6 + k];
    double C2[4];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) acc += T[3 * i + k] * S[3 * k + l] * T[3 * j + l];
            C2[2 * i + j] = acc;
        }
    double s00 = C2[0] + 0.3, s01 = C2[1], s11 = C2[3] + 0.3;
    double det = s00 * s11 - s01 * s01;
    out[0] = fx * xz + c->cx;
    out[1] = fy * yz + c->cy;
    out[2] = p[2];
    out[3] = s00; out[4] = s01; out[5] = s11;
    out[6] = s11 / det;        /* a */
    out[7] = -2.0 * s01 / det; /* b (the cross term's full coefficient) */
    out[8] = s00 / det;        /* c */
    out[9] = det;
}

/*
 * Rounding scale of a single-precision evaluation of the 2x3 factor
 * U = J W Q diag(s) of Sigma' - 0.3 I = U U^T (test tolerance only, not part of
 * the render): each entry of row r is a sum of products whose magnitudes are
 * bounded by |J_r| max(s), so an FP32 evaluation errs by a few units in the
 * last place of that size, whatever cancellation the sum has. Returns
 * |J_0| |J_1| max(s)^2.
 */
static double u_rows_scale(const float* mf, const float* sf, const orc_camera* c)
{
    double p[3];
    for (int i = 0; i < 3; i++)
        p[i] = (double)c->R[3 * i] * mf[0] + (double)c->R[3 * i + 1] * mf[1] + (double)c->R[3 * i + 2] * mf[2] + c->t[i];
    double limx = 1.3 * (0.5 * c->width / (double)c->fx), limy = 1.3 * (0.5 * c->height / (double)c->fy);
    double xz = p[0] / p[2], yz = p[1] / p[2];
    double cxz = xz < -limx ? -limx : (xz > limx ? limx : xz);
    double cyz = yz < -limy ? -limy : (yz > limy ? limy : yz);
    double smax = sf[0] > sf[1] ? sf[0] : sf[1];
    if (sf[2] > smax) smax = sf[2];
    double j0 = fabs((double)c->fx / p[2]) * sqrt(1.0 + cxz * cxz);
    double j1 = fabs((double)c->fy / p[2]) * sqrt(1.0 + cyz * cyz);
    return j0 * j1 * smax * smax;
}

/* View-dependent colour: sum_k Y_k(d) SH_k + 0.5, clamped to [0,1]. sh is [16][3]. */
void orc_sh_colour(const float* mf, const double* sh, int deg, const orc_camera* c, double* rgb)
{
    double campos[3];
    for (int j = 0; j < 3; j++) /* camera centre = -R^T t */
        campos[j] = -((double)c->R[j] * c->t[0] + (double)c->R[3 + j] * c->t[1] + (double)c->R[6 + j] * c->t[2]);
    double d[3] = {mf[0] - campos[0], mf[1] - campos[1], mf[2] - campos[2]};
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Y[16];
    orc_sh_basis(d[0] / n, d[1] / n, d[2] / n, Y);
    int nk = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.5;
        for (int k = 0; k < nk; k++) acc += Y[k] * sh[3 * k + ch];
        rgb[ch] = acc < 0 ? 0 : (acc > 1 ? 1 : acc);
    }
}

/* Eq. (24): I(P) = floor(P 2^23 log2(e) + 2^23 (127 - sigma)), reinterpreted as FP32. */
double orc_fast_exp64(double P)
{
    double I = floor(P * 8388608.0 * 1.4426950408889634 + 8388608.0 * (127.0 - ORC_SIGMA));
    if (I < 0) I = 0;
    uint32_t bits = (uint32_t)(int64_t)I;
    float f;
    memcpy(&f, &bits, 4);
    return (double)f;
}

/* Eq. (24) as one FP32 fused multiply-add followed by truncation toward zero. */
double orc_fast_exp32(float P)
{
    float y = fmaf(P, 12102203.0f, 1064970048.0f);
    int32_t I = (int32_t)y;
    if (I < 0) I = 0;
    uint32_t bits = (uint32_t)I;
    float f;
    memcpy(&f, &bits, 4);
    return (double)f;
}

/* ------------------------------------------------------------------------- */
/* Tiled render.                                                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    double key; /* depth order key: FP64 depth (exact) or quantized depth (RoofGS) */
    int64_t idx;
} orc_ord;

static int cmp_ord(const void* pa, const void* pb)
{
    const orc_ord* a = (const orc_ord*)pa;
    const orc_ord* b = (const orc_ord*)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/*
 * Render the listed tiles (all tiles if tiles == NULL) of one camera.
 *
 * means [n][3], quats [n][4] (w,x,y,z), scales [n][3] (activated), op [n]
 * (o in exact mode, log o in RoofGS mode), sh [n][16][3] FP64 coefficients.
 * img [3][H][W] receives C + T bg for every pixel of the rendered tiles.
 * diag (optional) [H][W][4] receives, per pixel (test tolerances, not part of
 * the render):
 *   [0] sum over contributing pairs of T_i alpha_i E_i, where E_i estimates the
 *       absolute FP32 rounding error of the pair's exponent (see below);
 *   [1] the sum of 2 T_i max(alpha_i, 1/255) over the pairs whose skip
 *       decision lies within E_i + slack of the 1/255 threshold (0 if none):
 *       the most the colour can jump if a single-precision renderer takes such
 *       a decision the other way;
 *   [2] the transmittance T_i before the first pair whose stop decision lies
 *       within the accumulated error of log T (sum of (alpha E + 2^-23) /
 *       (1 - alpha) over the blended pairs) + slack of the 1e-4 threshold;
 *   [3] number of pairs that contributed.
 * E_i is the first-order size of FP32 rounding in the exponent as the two
 * modes evaluate it:
 *   RoofGS mode (the folded polynomial of Eqs. (13)-(16) in tile-local
 *   coordinates, single-precision projected mean):
 *   E_i = 2^-23 (S_i + G_i (|u|+|v|) + 16), S_i the sum of the absolute terms of
 *   the exponent in tile-local coordinates, G_i = |grad_mu q|; slack 1e-5;
 *   exact mode (Eq. (10) as -1/2 (a' t^2 + dy^2 / Sigma'_yy) with
 *   t = dx - (Sigma'_xy / Sigma'_yy) dy, a' = Sigma'_yy / det, the mean carried
 *   at twice single precision):
 *   E_i = 2^-23 (32 |p| + 16 a' |t| (|dx| + |c| |dy| + |dy| g / Sigma'_yy) + 16),
 *   c = Sigma'_xy / Sigma'_yy, g = u_rows_scale(); slack 1e-6.
 * Returns the number of (tile, Gaussian) entries of the listed tiles, or -1.
 */
int64_t orc_render(int64_t n, const float* means, const float* quats, const float* scales,
                   const float* op, const double* sh, int sh_deg, const orc_camera* cam,
                   int mode, int32_t tile_w, int32_t tile_h, int exp_kind,
                   const int32_t* tiles, int64_t n_tiles, double* img, double* diag)
{
    orc_layout L;
    if (orc_layout_compute(cam, tile_w, tile_h, &L) != 0) return -1;
    const int W = cam->width, H = cam->height;
    int64_t NT = (int64_t)L.tiles_x * L.tiles_y;

    orc_bin* bins = (orc_bin*)malloc(sizeof(orc_bin) * (size_t)(n > 0 ? n : 1));
    char* want = (char*)calloc((size_t)NT, 1);
    if (!bins || !want) { free(bins); free(want); return -1; }
    if (tiles) {
        for (int64_t i = 0; i < n_tiles; i++)
            if (tiles[i] >= 0 && tiles[i] < NT) want[tiles[i]] = 1;
    } else {
        memset(want, 1, (size_t)NT);
    }
    for (int64_t i = 0; i < n; i++)
        bin32(means + 3 * i, quats + 4 * i, scales + 3 * i, op[i], mode, cam, &L, &bins[i]);

    /* CSR lists of the wanted tiles */
    int64_t* cnt = (int64_t*)calloc((size_t)NT + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        if (!bins[i].vis) continue;
        for (int ty = bins[i].ty0; ty <= bins[i].ty1; ty++) {
            int32_t ta, tb;
            if (!row_range(&bins[i], mode, &L, ty, &ta, &tb)) continue;
            for (int tx = ta; tx <= tb; tx++) {
                int64_t t = (int64_t)ty * L.tiles_x + tx;
                if (want[t]) cnt[t + 1]++;
            }
        }
    }
    for (int64_t t = 0; t < NT; t++) cnt[t + 1] += cnt[t];
    int64_t total = cnt[NT];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(NT + 1));
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(NT + 1));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    for (int64_t i = 0; i < n; i++) {
        if (!bins[i].vis) continue;
        for (int ty = bins[i].ty0; ty <= bins[i].ty1; ty++) {
            int32_t ta, tb;
            if (!row_range(&bins[i], mode, &L, ty, &ta, &tb)) continue;
            for (int tx = ta; tx <= tb; tx++) {
                int64_t t = (int64_t)ty * L.tiles_x + tx;
                if (want[t]) list[fill[t]++] = i;
            }
        }
    }

    /* FP64 per-Gaussian quantities, only for Gaussians that some wanted tile uses */
    char* used = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t e = 0; e < total; e++) used[list[e]] = 1;
    orc_g64* g = (orc_g64*)malloc(sizeof(orc_g64) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        if (!used[i]) continue;
        double pr[10];
        orc_project64(means + 3 * i, quats + 4 * i, scales + 3 * i, cam, pr);
        g[i].u = pr[0]; g[i].v = pr[1]; g[i].z = pr[2];
        g[i].s00 = pr[3]; g[i].s01 = pr[4]; g[i].s11 = pr[5];
        g[i].a = pr[6]; g[i].b = pr[7]; g[i].c = pr[8];
        g[i].gg = (mode == ORC_EXACT) ? u_rows_scale(means + 3 * i, scales + 3 * i, cam) : 0.0;
        g[i].op = op[i];
        orc_sh_colour(means + 3 * i, sh + 48 * i, sh_deg, cam, g[i].rgb);
    }

    const double eps32 = 1.0 / 8388608.0;
    orc_ord* ord = NULL;
    int64_t ord_cap = 0;
    for (int64_t t = 0; t < NT; t++) {
        if (!want[t]) continue;
        int64_t len = cnt[t + 1] - cnt[t];
        if (len > ord_cap) {
            free(ord);
            ord_cap = len;
            ord = (orc_ord*)malloc(sizeof(orc_ord) * (size_t)ord_cap);
        }
        for (int64_t e = 0; e < len; e++) {
            int64_t i = list[cnt[t] + e];
            ord[e].idx = i;
            ord[e].key = (mode == ORC_EXACT) ? g[i].z : (double)bins[i].qd;
        }
        qsort(ord, (size_t)len, sizeof(orc_ord), cmp_ord);
        int tx = (int)(t % L.tiles_x), ty = (int)(t / L.tiles_x);
        int x0 = tx * tile_w, y0 = ty * tile_h;
        for (int py = y0; py < y0 + tile_h && py < H; py++)
            for (int px = x0; px < x0 + tile_w && px < W; px++) {
                double T = 1.0, C[3] = {0, 0, 0};
                double d0 = 0, d1 = 0, d2 = 0, d3 = 0, eacc = 0;
                for (int64_t e = 0; e < len; e++) {
                    const orc_g64* G = &g[ord[e].idx];
                    double dx = px - G->u, dy = py - G->v;
                    double p = -0.5 * (G->a * dx * dx + G->b * dx * dy + G->c * dy * dy);
                    /* rounding-size estimate of a single-precision evaluation */
                    double E, slack;
                    if (mode == ORC_EXACT) {
                        double cc = G->s01 / G->s11;
                        double t = dx - cc * dy;
                        E = eps32 * (32.0 * fabs(p) +
                                     16.0 * G->a * fabs(t) * (fabs(dx) + fabs(cc) * fabs(dy) + fabs(dy) * G->gg / G->s11) +
                                     16.0);
                        slack = 1e-6;
                    } else {
                        double lx = px - x0, ly = py - y0, lu = G->u - x0, lv = G->v - y0;
                        double ax = fabs(lx) + fabs(lu), ay = fabs(ly) + fabs(lv);
                        double S = fabs(G->a) * ax * ax + fabs(G->b) * ax * ay + fabs(G->c) * ay * ay;
                        double gx = 2 * G->a * dx + G->b * dy, gy = G->b * dx + 2 * G->c * dy;
                        double Gm = sqrt(gx * gx + gy * gy);
                        E = eps32 * (S + Gm * (fabs(G->u) + fabs(G->v)) + 16.0);
                        slack = 1e-5;
                    }
                    double alpha, margin;
                    if (mode == ORC_EXACT) {
                        if (p > 0) continue;
                        double at = G->op * exp(p);
                        margin = log(255.0 * at);
                        alpha = at < 0.99 ? at : 0.99;
                        if (alpha < 1.0 / 255.0) {
                            if (fabs(margin) < E + slack) d1 += 2.0 * T / 255.0;
                            continue;
                        }
                    } else {
                        double P = p + G->op; /* Eq. (17) */
                        margin = P + ORC_LN255;
                        if (P < -ORC_LN255) { /* outside the range of Eq. (23) */
                            if (fabs(margin) < E + slack) d1 += 2.0 * T / 255.0;
                            continue;
                        }
                        double at;
                        if (exp_kind == ORC_EXP_FAST64) at = orc_fast_exp64(P);
                        else if (exp_kind == ORC_EXP_FAST32) at = orc_fast_exp32((float)P);
                        else at = exp(P);
                        alpha = at < 0.99 ? at : 0.99; /* Eq. (25) */
                    }
                    if (fabs(margin) < E + slack) d1 += 2.0 * T * (alpha > 1.0 / 255 ? alpha : 1.0 / 255);
                    double Tn = T * (1.0 - alpha);
                    eacc += (alpha * E + eps32) / (1.0 - alpha);
                    if (d2 == 0 && fabs(log(Tn / 1e-4)) < eacc + slack) d2 = T;
                    if (Tn < 1e-4) break; /* stop without adding this pair */
                    for (int ch = 0; ch < 3; ch++) C[ch] += G->rgb[ch] * alpha * T;
                    d0 += T * alpha * E;
                    d3 += 1;
                    T = Tn;
                }
                for (int ch = 0; ch < 3; ch++)
                    img[(int64_t)ch * H * W + (int64_t)py * W + px] = C[ch] + T * (double)cam->bg[ch];
                if (diag) {
                    double* dp = diag + ((int64_t)py * W + px) * 4;
                    dp[0] = d0; dp[1] = d1; dp[2] = d2; dp[3] = d3;
                }
            }
    }
    free(ord);
    free(g);
    free(used);
    free(list);
    free(fill);
    free(cnt);
    free(want);
    free(bins);
    return total;
}

/*
 * Sorted (key, value) entries of the whole frame, as the FP32 binning path
 * defines them: one entry per (tile, Gaussian) of each Gaussian's tile
 * rectangle, key = tile|float-depth (exact, 64-bit) or tile|q_d (RoofGS,
 * 32-bit), value = Gaussian index, ascending by (key, index).
 * If keys/vals are NULL or cap is too small, only the count is returned.
 * Also returns per-tile [start, end) ranges into ranges[2*NT] if given.
 */
typedef struct {
    uint64_t key;
    uint32_t val;
} orc_kv;

static int cmp_kv(const void* pa, const void* pb)
{
    const orc_kv* a = (const orc_kv*)pa;
    const orc_kv* b = (const orc_kv*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->val > b->val) - (a->val < b->val);
}

int64_t orc_keys(int64_t n, const float* means, const float* quats, const float* scales,
                 const float* op, const orc_camera* cam, int mode, int32_t tile_w, int32_t tile_h,
                 uint64_t* keys, uint32_t* vals, int64_t cap, uint32_t* ranges, int32_t* binout)
{
    orc_layout L;
    if (orc_layout_compute(cam, tile_w, tile_h, &L) != 0) return -1;
    int64_t total = 0;
    orc_bin* bins = (orc_bin*)malloc(sizeof(orc_bin) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        bin32(means + 3 * i, quats + 4 * i, scales + 3 * i, op[i], mode, cam, &L, &bins[i]);
        int64_t ni = 0;
        if (bins[i].vis)
            for (int ty = bins[i].ty0; ty <= bins[i].ty1; ty++) {
                int32_t ta, tb;
                if (row_range(&bins[i], mode, &L, ty, &ta, &tb)) ni += tb - ta + 1;
            }
        total += ni;
        if (binout) {
            int32_t* o = binout + 7 * i;
            o[0] = bins[i].vis; o[1] = bins[i].tx0; o[2] = bins[i].ty0;
            o[3] = bins[i].tx1; o[4] = bins[i].ty1; o[5] = (int32_t)bins[i].qd;
            o[6] = (int32_t)ni;
        }
    }
    if (keys && vals && total <= cap) {
        orc_kv* kv = (orc_kv*)malloc(sizeof(orc_kv) * (size_t)(total > 0 ? total : 1));
        int64_t e = 0;
        for (int64_t i = 0; i < n; i++) {
            if (!bins[i].vis) continue;
            for (int ty = bins[i].ty0; ty <= bins[i].ty1; ty++) {
                int32_t ta, tb;
                if (!row_range(&bins[i], mode, &L, ty, &ta, &tb)) continue;
                for (int tx = ta; tx <= tb; tx++) {
                    kv[e].key = entry_key(&bins[i], mode, &L, ty * L.tiles_x + tx);
                    kv[e].val = (uint32_t)i;
                    e++;
                }
            }
        }
        qsort(kv, (size_t)total, sizeof(orc_kv), cmp_kv);
        for (int64_t k = 0; k < total; k++) { keys[k] = kv[k].key; vals[k] = kv[k].val; }
        if (ranges) {
            int64_t NT = (int64_t)L.tiles_x * L.tiles_y;
            memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)NT);
            for (int64_t k = 0; k < total; k++) {
                uint64_t tile = (mode == ORC_EXACT) ? (kv[k].key >> 32)
                                                    : (L.b_d >= 32 ? 0 : (kv[k].key >> L.b_d));
                if (k == 0 || tile != ((mode == ORC_EXACT) ? (kv[k - 1].key >> 32)
                                                         : (L.b_d >= 32 ? 0 : (kv[k - 1].key >> L.b_d))))
                    ranges[2 * tile] = (uint32_t)k;
                ranges[2 * tile + 1] = (uint32_t)(k + 1);
            }
        }
        free(kv);
    }
    free(bins);
    return total;
}

/* Layout query for tests: tiles_x, tiles_y, b_t, b_d, qmax, depth_scale bits. */
int orc_layout_query(const orc_camera* cam, int32_t tile_w, int32_t tile_h, int64_t* out)
{
    orc_layout L;
    if (orc_layout_compute(cam, tile_w, tile_h, &L) != 0) return -1;
    out[0] = L.tiles_x; out[1] = L.tiles_y; out[2] = L.b_t; out[3] = L.b_d;
    out[4] = L.qmax; out[5] = f32_bits(L.depth_scale);
    return 0;
}

/* log o in FP64, rounded to FP32: the stored opacity of RoofGS mode. */
void orc_log_opacity(int64_t n, const float* o, float* out)
{
    for (int64_t i = 0; i < n; i++) out[i] = (float)log((double)o[i]);
}

/* Vectorised Eq. (24) for tests: kind ORC_EXP_FAST64 or ORC_EXP_FAST32. */
void orc_fast_exp_many(int64_t n, const double* P, double* out, int kind)
{
    for (int64_t i = 0; i < n; i++)
        out[i] = (kind == ORC_EXP_FAST32) ? orc_fast_exp32((float)P[i]) : orc_fast_exp64(P[i]);
}

/* ------------------------------------------------------------------------- */
/* FP64 gradient of the exact-mode render.                                      */
/* ------------------------------------------------------------------------- */

/*
 * The per-Gaussian map of the exact mode in complex arithmetic, for
 * complex-step differentiation (Squire and Trapp 1998: for a real-analytic f,
 * f'(x) = Im f(x + i h) / h up to rounding, with no difference of nearby
 * values, so h = 1e-30 gives the derivative to FP64 precision). The
 * definitions are those of orc_project64 and orc_sh_colour: mean, raw
 * quaternion and scale -> (u, v, a, b, c) of Eq. (10); mean -> the raw colour
 * sum_k Y_k(d) SH_k + 0.5 before the clamp. The tangent clamp compares real
 * parts (a piecewise map: the derivative of the branch taken).
 */
typedef double _Complex cplx;

static cplx cmin_re(cplx a, double lim) { return creal(a) > lim ? (cplx)lim : a; }
static cplx cmax_re(cplx a, double lim) { return creal(a) < lim ? (cplx)lim : a; }

static void proj_cplx(const cplx* m, const cplx* q, const cplx* s, const orc_camera* c, cplx* out)
{
    double R[9];
    for (int i = 0; i < 9; i++) R[i] = c->R[i];
    cplx p[3];
    for (int i = 0; i < 3; i++) p[i] = R[3 * i] * m[0] + R[3 * i + 1] * m[1] + R[3 * i + 2] * m[2] + (double)c->t[i];
    cplx nq = csqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    cplx w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
    cplx Q[9];
    Q[0] = 1.0 - 2.0 * (y * y + z * z); Q[1] = 2.0 * (x * y - w * z);       Q[2] = 2.0 * (x * z + w * y);
    Q[3] = 2.0 * (x * y + w * z);       Q[4] = 1.0 - 2.0 * (x * x + z * z); Q[5] = 2.0 * (y * z - w * x);
    Q[6] = 2.0 * (x * z - w * y);       Q[7] = 2.0 * (y * z + w * x);       Q[8] = 1.0 - 2.0 * (x * x + y * y);
    cplx S[9]; /* Sigma = Q diag(s)^2 Q^T */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++) acc += Q[3 * i + k] * s[k] * s[k] * Q[3 * j + k];
            S[3 * i + j] = acc;
        }
    double fx = c->fx, fy = c->fy;
    double limx = 1.3 * (0.5 * c->width / fx), limy = 1.3 * (0.5 * c->height / fy);
    cplx xz = p[0] / p[2], yz = p[1] / p[2];
    cplx cxz = cmax_re(cmin_re(xz, limx), -limx), cyz = cmax_re(cmin_re(yz, limy), -limy);
    cplx J[6] = {fx / p[2], 0, -fx * cxz / p[2], 0, fy / p[2], -fy * cyz / p[2]};
    cplx T[6];
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++) T[3 * i + k] = J[3 * i] * R[k] + J[3 * i + 1] * R[3 + k] + J[3 * i + 2] * R[6 + k];
    cplx C2[4];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) acc += T[3 * i + k] * S[3 * k + l] * T[3 * j + l];
            C2[2 * i + j] = acc;
        }
    cplx s00 = C2[0] + 0.3, s01 = C2[1], s11 = C2[3] + 0.3;
    cplx det = s00 * s11 - s01 * s01;
    out[0] = fx * xz + (double)c->cx;
    out[1] = fy * yz + (double)c->cy;
    out[2] = s11 / det;
    out[3] = -2.0 * s01 / det;
    out[4] = s00 / det;
}

static void sh_basis_cplx(cplx x, cplx y, cplx z, cplx* Y)
{
    const double pi = 3.14159265358979323846;
    Y[0] = 0.5 * sqrt(1.0 / pi);
    double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = k1 * y;
    Y[2] = k1 * z;
    Y[3] = k1 * x;
    double k2a = 0.5 * sqrt(15.0 / pi), k20 = 0.25 * sqrt(5.0 / pi), k22 = 0.25 * sqrt(15.0 / pi);
    Y[4] = k2a * x * y;
    Y[5] = k2a * y * z;
    Y[6] = k20 * (3.0 * z * z - 1.0);
    Y[7] = k2a * x * z;
    Y[8] = k22 * (x * x - y * y);
    double k33 = 0.25 * sqrt(35.0 / (2.0 * pi)), k32 = 0.5 * sqrt(105.0 / pi);
    double k31 = 0.25 * sqrt(21.0 / (2.0 * pi)), k30 = 0.25 * sqrt(7.0 / pi), k32b = 0.25 * sqrt(105.0 / pi);
    Y[9] = k33 * y * (3.0 * x * x - y * y);
    Y[10] = k32 * x * y * z;
    Y[11] = k31 * y * (5.0 * z * z - 1.0);
    Y[12] = k30 * z * (5.0 * z * z - 3.0);
    Y[13] = k31 * x * (5.0 * z * z - 1.0);
    Y[14] = k32b * z * (x * x - y * y);
    Y[15] = k33 * x * (x * x - 3.0 * y * y);
}

/* raw colour (before the [0, 1] clamp) of one Gaussian; sh is [16][3] */
static void colour_raw_cplx(const cplx* m, const double* sh, int deg, const orc_camera* c, cplx* raw)
{
    double campos[3];
    for (int j = 0; j < 3; j++)
        campos[j] = -((double)c->R[j] * c->t[0] + (double)c->R[3 + j] * c->t[1] + (double)c->R[6 + j] * c->t[2]);
    cplx d[3] = {m[0] - campos[0], m[1] - campos[1], m[2] - campos[2]};
    cplx nd = csqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    cplx Y[16];
    sh_basis_cplx(d[0] / nd, d[1] / nd, d[2] / nd, Y);
    int nk = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ch++) {
        cplx acc = 0.5;
        for (int k = 0; k < nk; k++) acc += Y[k] * sh[3 * k + ch];
        raw[ch] = acc;
    }
}

/*
 * Gradient of L = sum(dL_dimg * img) for the exact-mode image of orc_render
 * (all tiles), with respect to the FP32 inputs: means [n][3], scales [n][3]
 * (activated), quats [n][4] (raw, normalised inside), opacities [n], sh
 * [n][16][3]. Outputs are FP64 and fully written.
 *
 * Per pixel (Sec. III-D, Eq. (7)): C = sum_i c_i alpha_i T_i + T_N bg with
 * T_i = prod_{j<i} (1 - alpha_j) over the pairs the forward blends (same skip
 * and stop rules, same FP64 depth order). Walking the pairs back to front with
 * R_i = sum_{j>i} c_j alpha_j T_j + T_N bg (the colour behind pair i):
 *   dC/dc_i = alpha_i T_i,   dC/dalpha_i = c_i T_i - R_i / (1 - alpha_i);
 * alpha = min(0.99, o e^p) (Eqs. (11)-(12)): below the clamp dalpha/do = e^p,
 * dalpha/dp = alpha, at the clamp both are 0; p = -1/2 (a dx^2 + b dx dy +
 * c dy^2) (Eq. (10)) with dx = x - u, dy = y - v gives dp/du = a dx + b dy / 2,
 * dp/dv = b dx / 2 + c dy, dp/da = -dx^2 / 2, dp/db = -dx dy / 2,
 * dp/dc = -dy^2 / 2. Per Gaussian, the sums over its pixels go through the
 * Jacobian of the map (mean, quaternion, scale) -> (u, v, a, b, c) and mean ->
 * raw colour, taken by complex steps; the clamp of the colour to [0, 1] passes
 * no gradient outside (0, 1); dL/dSH_k = Y_k(d) dL/draw.
 * Returns 0, or -1 on a bad layout or allocation failure.
 */
int orc_backward(int64_t n, const float* means, const float* quats, const float* scales, const float* opac,
                 const double* sh, int sh_deg, const orc_camera* cam, int32_t tile_w, int32_t tile_h,
                 const double* dL_dimg, double* dmeans, double* dscales, double* dquats, double* dopac, double* dsh)
{
    orc_layout L;
    if (orc_layout_compute(cam, tile_w, tile_h, &L) != 0) return -1;
    const int W = cam->width, H = cam->height;
    const int64_t NT = (int64_t)L.tiles_x * L.tiles_y;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    memset(dmeans, 0, sizeof(double) * 3 * nn);
    memset(dscales, 0, sizeof(double) * 3 * nn);
    memset(dquats, 0, sizeof(double) * 4 * nn);
    memset(dopac, 0, sizeof(double) * nn);
    memset(dsh, 0, sizeof(double) * 48 * nn);

    orc_bin* bins = (orc_bin*)malloc(sizeof(orc_bin) * nn);
    int64_t* cnt = (int64_t*)calloc((size_t)NT + 1, sizeof(int64_t));
    if (!bins || !cnt) { free(bins); free(cnt); return -1; }
    for (int64_t i = 0; i < n; i++) bin32(means + 3 * i, quats + 4 * i, scales + 3 * i, opac[i], ORC_EXACT, cam, &L, &bins[i]);
    for (int64_t i = 0; i < n; i++) {
        if (!bins[i].vis) continue;
        for (int ty = bins[i].ty0; ty <= bins[i].ty1; ty++)
            for (int tx = bins[i].tx0; tx <= bins[i].tx1; tx++) cnt[(int64_t)ty * L.tiles_x + tx + 1]++;
    }
    for (int64_t t = 0; t < NT; t++) cnt[t + 1] += cnt[t];
    const int64_t total = cnt[NT];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(NT + 1));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    orc_g64* g = (orc_g64*)malloc(sizeof(orc_g64) * nn);
    double* gimg = (double*)calloc(nn * 9, sizeof(double)); /* per Gaussian: d(u, v, a, b, c), d(o), d(rgb) */
    if (!fill || !list || !g || !gimg) { free(bins); free(cnt); free(fill); free(list); free(g); free(gimg); return -1; }
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(NT + 1));
    for (int64_t i = 0; i < n; i++) {
        if (!bins[i].vis) continue;
        for (int ty = bins[i].ty0; ty <= bins[i].ty1; ty++)
            for (int tx = bins[i].tx0; tx <= bins[i].tx1; tx++) list[fill[(int64_t)ty * L.tiles_x + tx]++] = i;
    }
    for (int64_t i = 0; i < n; i++) {
        if (!bins[i].vis) continue;
        double pr[10];
        orc_project64(means + 3 * i, quats + 4 * i, scales + 3 * i, cam, pr);
        g[i].u = pr[0]; g[i].v = pr[1]; g[i].z = pr[2];
        g[i].a = pr[6]; g[i].b = pr[7]; g[i].c = pr[8];
        g[i].op = opac[i];
        orc_sh_colour(means + 3 * i, sh + 48 * i, sh_deg, cam, g[i].rgb);
    }

    typedef struct { int64_t i; double alpha, T, e, dx, dy; int clamped; } pair_t;
    orc_ord* ord = NULL;
    pair_t* pr = NULL;
    int64_t cap = 0;
    for (int64_t t = 0; t < NT; t++) {
        int64_t len = cnt[t + 1] - cnt[t];
        if (len == 0) continue;
        if (len > cap) {
            free(ord); free(pr);
            cap = len;
            ord = (orc_ord*)malloc(sizeof(orc_ord) * (size_t)cap);
            pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)cap);
        }
        for (int64_t e = 0; e < len; e++) {
            ord[e].idx = list[cnt[t] + e];
            ord[e].key = g[ord[e].idx].z;
        }
        qsort(ord, (size_t)len, sizeof(orc_ord), cmp_ord);
        int tx = (int)(t % L.tiles_x), ty = (int)(t / L.tiles_x);
        for (int py = ty * tile_h; py < ty * tile_h + tile_h && py < H; py++)
            for (int px = tx * tile_w; px < tx * tile_w + tile_w && px < W; px++) {
                /* forward: the blended pairs of this pixel */
                double T = 1.0;
                int64_t np_ = 0;
                for (int64_t e = 0; e < len; e++) {
                    const orc_g64* G = &g[ord[e].idx];
                    double dx = px - G->u, dy = py - G->v;
                    double p = -0.5 * (G->a * dx * dx + G->b * dx * dy + G->c * dy * dy);
                    if (p > 0) continue;
                    double ex = exp(p), at = G->op * ex;
                    double alpha = at < 0.99 ? at : 0.99;
                    if (alpha < 1.0 / 255.0) continue;
                    double Tn = T * (1.0 - alpha);
                    if (Tn < 1e-4) break;
                    pr[np_].i = ord[e].idx; pr[np_].alpha = alpha; pr[np_].T = T; pr[np_].e = ex;
                    pr[np_].dx = dx; pr[np_].dy = dy; pr[np_].clamped = !(at < 0.99);
                    np_++;
                    T = Tn;
                }
                double Gc[3], R[3];
                for (int ch = 0; ch < 3; ch++) {
                    Gc[ch] = dL_dimg[(int64_t)ch * H * W + (int64_t)py * W + px];
                    R[ch] = T * (double)cam->bg[ch];
                }
                /* backward: back to front */
                for (int64_t k = np_ - 1; k >= 0; k--) {
                    const pair_t* P = &pr[k];
                    const orc_g64* G = &g[P->i];
                    double* gi = gimg + 9 * P->i;
                    double dal = 0;
                    for (int ch = 0; ch < 3; ch++) {
                        gi[6 + ch] += Gc[ch] * P->alpha * P->T;
                        dal += Gc[ch] * (G->rgb[ch] * P->T - R[ch] / (1.0 - P->alpha));
                        R[ch] += G->rgb[ch] * P->alpha * P->T;
                    }
                    if (P->clamped) continue;
                    gi[5] += dal * P->e;
                    double dp = dal * P->alpha;
                    gi[0] += dp * (G->a * P->dx + 0.5 * G->b * P->dy);
                    gi[1] += dp * (0.5 * G->b * P->dx + G->c * P->dy);
                    gi[2] += dp * (-0.5 * P->dx * P->dx);
                    gi[3] += dp * (-0.5 * P->dx * P->dy);
                    gi[4] += dp * (-0.5 * P->dy * P->dy);
                }
            }
    }

    /* per Gaussian: through (u, v, a, b, c) and the raw colour to the inputs */
    const double h = 1e-30;
    for (int64_t i = 0; i < n; i++) {
        if (!bins[i].vis) continue;
        const double* gi = gimg + 9 * i;
        dopac[i] = gi[5];
        cplx m0[3], q0[4], s0[3], raw[3];
        for (int k = 0; k < 3; k++) { m0[k] = means[3 * i + k]; s0[k] = scales[3 * i + k]; }
        for (int k = 0; k < 4; k++) q0[k] = quats[4 * i + k];
        colour_raw_cplx(m0, sh + 48 * i, sh_deg, cam, raw);
        double draw[3];
        for (int ch = 0; ch < 3; ch++) {
            double r = creal(raw[ch]);
            draw[ch] = (r > 0.0 && r < 1.0) ? gi[6 + ch] : 0.0;
        }
        /* dL/dSH_k = Y_k dL/draw */
        {
            double campos[3];
            for (int j = 0; j < 3; j++)
                campos[j] = -((double)cam->R[j] * cam->t[0] + (double)cam->R[3 + j] * cam->t[1] +
                              (double)cam->R[6 + j] * cam->t[2]);
            double d[3] = {means[3 * i] - campos[0], means[3 * i + 1] - campos[1], means[3 * i + 2] - campos[2]};
            double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double Y[16];
            orc_sh_basis(d[0] / nd, d[1] / nd, d[2] / nd, Y);
            int nk = (sh_deg + 1) * (sh_deg + 1);
            for (int k = 0; k < nk; k++)
                for (int ch = 0; ch < 3; ch++) dsh[48 * i + 3 * k + ch] = Y[k] * draw[ch];
        }
        for (int j = 0; j < 10; j++) { /* inputs: mean 0-2, quaternion 3-6, scale 7-9 */
            cplx m[3], q[4], s[3], out[5];
            for (int k = 0; k < 3; k++) { m[k] = m0[k]; s[k] = s0[k]; }
            for (int k = 0; k < 4; k++) q[k] = q0[k];
            if (j < 3) m[j] += h * _Complex_I;
            else if (j < 7) q[j - 3] += h * _Complex_I;
            else s[j - 7] += h * _Complex_I;
            proj_cplx(m, q, s, cam, out);
            double acc = 0;
            for (int o = 0; o < 5; o++) acc += gi[o] * cimag(out[o]) / h;
            if (j < 3) {
                colour_raw_cplx(m, sh + 48 * i, sh_deg, cam, raw);
                for (int ch = 0; ch < 3; ch++) acc += draw[ch] * cimag(raw[ch]) / h;
                dmeans[3 * i + j] = acc;
            } else if (j < 7) {
                dquats[4 * i + j - 3] = acc;
            } else {
                dscales[3 * i + j - 7] = acc;
            }
        }
    }
    free(ord); free(pr); free(gimg); free(g); free(list); free(fill); free(cnt); free(bins);
    return 0;
}
