/*
 * FP64 CPU oracle of the differentiable tile-based Gaussian splatting
 * rasterizer that the joint pose and primitive optimisation runs every
 * iteration (Sec. 4.3; the paper builds on the 3DGS image-formation model,
 * Sec. 5, and states no rasterizer equations, so each step below is that model
 * written out as mathematics).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code, header, constant or table with the CUDA
 * library; the two meet only in the seeded inputs they both consume.
 *
 * Readings taken where the paper is silent (all configurable through `cfg`):
 *   near-plane cull z <= near; screen-space dilation Sigma2D + dil*I with the
 *   opacity unchanged; Jacobian guard band |x/z| <= 1.3 (W/2)/fx (and for y);
 *   3-sigma radius from the largest eigenvalue with the 0.1 floor; tile rect
 *   [floor((u-r)/T), floor((u+r+T-1)/T)) clamped to the grid; pixel (i, j)
 *   sampled at (i+0.5, j+0.5); alpha = min(alpha_max, o*exp(power)), skipped if
 *   alpha < alpha_min or power > 0; compositing stops before the Gaussian that
 *   would take T below t_min; orthonormal real SH with the Condon-Shortley
 *   phase; colour = SH + 0.5 clamped at 0; dalpha/d(o*g) = 0 where alpha is
 *   clamped; pose gradient for a left perturbation T_cw <- exp(xi^) T_cw,
 *   xi = (rho, phi), without the SH view-direction path unless enabled.
 *
 * Every discrete decision records its margin. Items whose margin is below the
 * configured relative threshold are flagged ambiguous so tests can exclude
 * them: FP32 arithmetic on the GPU may legitimately take the other branch.
 *
 * cam[18] = R(9, row-major world->camera), t(3), fx, fy, cx, cy, width, height
 * cfg[18] = tile, sh_degree, near, dilation, alpha_min, alpha_max, t_min,
 *           bg(3), pose_grad_through_sh, margin_geo, margin_alpha, margin_T,
 *           margin_rect_px, margin_depth, mip_filter, alpha_rect
 * alpha_rect = 1: the tile rect is also bounded by the tiles the box of the
 * ellipse where o exp(-q/2) reaches alpha_min overlaps: x within u +- hx,
 * hx = sqrt(2 ln(o / alpha_min) Sigma2D_xx) (y likewise), tiles
 * [floor((u - hx)/T), floor((u + hx)/T) + 1); the 3-sigma rect and this one
 * are intersected, and an opacity below alpha_min lists the item nowhere. A
 * pixel centre where alpha reaches alpha_min lies in the box, so no composited
 * (pixel, Gaussian) pair is dropped: only list entries no pixel composites.
 * mip_filter = 1: the dilation acts as a 2-D low-pass filter that keeps the
 * splat's integral (the multi-scale filtering of Sec. 4.3): the opacity is
 * multiplied by sqrt(rho), rho = det(Sigma2D) / det(Sigma2D + dil I), with rho
 * floored at 1e-6 (a degenerate splat keeps a tiny, gradient-free weight).
 * margin_geo is relative (near plane, determinant, radius, guard band, colour
 * clamp); margin_rect_px is the distance in pixels of a tile-rect edge from a
 * tile boundary; margin_alpha and margin_T are relative; margin_depth flags a
 * pixel whose composited Gaussians include two with depths equal to within
 * that relative margin (their fp32 sort order may differ).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846

typedef struct {
    double R[9], t[3], fx, fy, cx, cy;
    int W, H;
} Cam;

typedef struct {
    int tile, sh_degree, pose_through_sh, mip, alpha_rect;
    double near_z, dil, a_min, a_max, t_min, bg[3], m_geo, m_alpha, m_T, m_rect, m_depth;
} Cfg;

static Cam read_cam(const double* c) {
    Cam k;
    for (int i = 0; i < 9; i++) k.R[i] = c[i];
    for (int i = 0; i < 3; i++) k.t[i] = c[9 + i];
    k.fx = c[12]; k.fy = c[13]; k.cx = c[14]; k.cy = c[15];
    k.W = (int)c[16]; k.H = (int)c[17];
    return k;
}

static Cfg read_cfg(const double* c) {
    Cfg g;
    g.tile = (int)c[0]; g.sh_degree = (int)c[1];
    g.near_z = c[2]; g.dil = c[3]; g.a_min = c[4]; g.a_max = c[5]; g.t_min = c[6];
    g.bg[0] = c[7]; g.bg[1] = c[8]; g.bg[2] = c[9];
    g.pose_through_sh = (int)c[10];
    g.m_geo = c[11]; g.m_alpha = c[12]; g.m_T = c[13]; g.m_rect = c[14]; g.m_depth = c[15];
    g.mip = (int)c[16];
    g.alpha_rect = (int)c[17];
    return g;
}

/* ---------------------------------------------------------------------------
 * Small dense helpers (3x3 row-major)
 * ------------------------------------------------------------------------- */
static void mat3_mul(const double* A, const double* B, double* C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}
static void mat3_T(const double* A, double* B) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[3 * i + j] = A[3 * j + i];
    memcpy(B, T, sizeof T);
}

/* rotation matrix of the unit quaternion (w, x, y, z) */
static void quat_to_rot(const double* q, double* R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static double dist_to_int(double v) { return fabs(v - nearbyint(v)); }

/* ---------------------------------------------------------------------------
 * Real spherical harmonics with the Condon-Shortley phase, degree <= 3.
 *
 * For a unit direction d = (x, y, z):
 *   Y_l^0  = K_l^0 q_l^0(z)
 *   Y_l^m  = sqrt(2) K_l^m q_l^m(z) Re((x + i y)^m)      m > 0
 *   Y_l^-m = sqrt(2) K_l^m q_l^m(z) Im((x + i y)^m)      m > 0
 * where q_l^m(z) = P_l^m(z) / (1 - z^2)^(m/2) (associated Legendre function
 * with the phase (-1)^m, divided by sin^m theta; a polynomial in z) and
 * K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). Coefficient index k = l^2 + l + m.
 * Evaluated on forward-mode dual numbers so the gradient w.r.t. d is exact.
 * ------------------------------------------------------------------------- */
typedef struct { double v, d[3]; } Dual;

static Dual dconst(double c) { Dual r = {c, {0, 0, 0}}; return r; }
static Dual dvar(double c, int i) { Dual r = {c, {0, 0, 0}}; r.d[i] = 1; return r; }
static Dual dadd(Dual a, Dual b) { Dual r; r.v = a.v + b.v; for (int i = 0; i < 3; i++) r.d[i] = a.d[i] + b.d[i]; return r; }
static Dual dsub(Dual a, Dual b) { Dual r; r.v = a.v - b.v; for (int i = 0; i < 3; i++) r.d[i] = a.d[i] - b.d[i]; return r; }
static Dual dmul(Dual a, Dual b) {
    Dual r; r.v = a.v * b.v;
    for (int i = 0; i < 3; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
static Dual dscale(Dual a, double s) { Dual r; r.v = a.v * s; for (int i = 0; i < 3; i++) r.d[i] = a.d[i] * s; return r; }

static double factorial(int n) { double f = 1; for (int i = 2; i <= n; i++) f *= i; return f; }

/* Y[16] values and dY[16][3] gradients w.r.t. (x, y, z) */
void or_sh_basis(int degree, const double* dir, double* Y, double* dY) {
    Dual x = dvar(dir[0], 0), y = dvar(dir[1], 1), z = dvar(dir[2], 2);
    Dual A[4], B[4];            /* Re, Im of (x + i y)^m */
    A[0] = dconst(1); B[0] = dconst(0);
    for (int m = 1; m <= 3; m++) {
        A[m] = dsub(dmul(x, A[m - 1]), dmul(y, B[m - 1]));
        B[m] = dadd(dmul(x, B[m - 1]), dmul(y, A[m - 1]));
    }
    Dual q[4][4];               /* q[l][m] */
    for (int m = 0; m <= 3; m++) {
        double dfact = 1;       /* (2m-1)!! */
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
        q[m][m] = dconst(((m & 1) ? -1.0 : 1.0) * dfact);
        if (m + 1 <= 3) q[m + 1][m] = dscale(dmul(z, q[m][m]), 2 * m + 1);
        for (int l = m + 2; l <= 3; l++)
            q[l][m] = dscale(dsub(dscale(dmul(z, q[l - 1][m]), 2 * l - 1),
                                  dscale(q[l - 2][m], l + m - 1)), 1.0 / (l - m));
    }
    for (int k = 0; k < 16; k++) { Y[k] = 0; dY[3 * k] = dY[3 * k + 1] = dY[3 * k + 2] = 0; }
    for (int l = 0; l <= degree; l++) {
        for (int m = -l; m <= l; m++) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2 * l + 1) / (4 * PI_D) * factorial(l - am) / factorial(l + am));
            Dual val;
            if (m == 0) val = dscale(q[l][0], K);
            else if (m > 0) val = dscale(dmul(q[l][am], A[am]), sqrt(2.0) * K);
            else val = dscale(dmul(q[l][am], B[am]), sqrt(2.0) * K);
            int k = l * l + l + m;
            Y[k] = val.v;
            for (int i = 0; i < 3; i++) dY[3 * k + i] = val.d[i];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Projection (EWA splatting + SH colour), one view.
 * ------------------------------------------------------------------------- */
typedef struct {
    int culled;
    double p[3], qn[4], qlen, Rq[9], s[3], Sig[9], Sc[9], J[6], S2[4], det;
    int clamp_x, clamp_y;
    double dir[3], dlen, d[3], Y[16], dY[48], raw[3];
    double o, rho, fmip; /* opacity before the filter factor; rho and sqrt(rho) (1 without the filter) */
    int rho_floor;       /* rho below its floor: no gradient through it */
} ProjState;

static void project_one(int64_t i, const double* mean_opa, const double* scale, const double* quat,
                        const double* sh, const Cam* k, const Cfg* g, ProjState* st,
                        double* mean2d, double* conic, double* opac, double* rgb, double* depth,
                        int32_t* rect, uint8_t* clampm, uint8_t* amb, uint8_t* side) {
    memset(st, 0, sizeof *st);
    st->culled = 1;
    double mu[3] = {mean_opa[4 * i], mean_opa[4 * i + 1], mean_opa[4 * i + 2]};
    double logit = mean_opa[4 * i + 3];
    for (int r = 0; r < 3; r++)
        st->p[r] = k->R[3 * r] * mu[0] + k->R[3 * r + 1] * mu[1] + k->R[3 * r + 2] * mu[2] + k->t[r];
    double x = st->p[0], y = st->p[1], z = st->p[2];
    uint8_t a = 0;
    if (fabs(z - g->near_z) < g->m_geo * fmax(1.0, fabs(z))) a |= 1;
    for (int c = 0; c < 4; c++) rect[4 * i + c] = 0;
    depth[i] = z;
    if (amb) amb[i] = a;
    if (!(z > g->near_z) || !isfinite(x) || !isfinite(y)) return;

    double q[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
    st->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int c = 0; c < 4; c++) st->qn[c] = q[c] / st->qlen;
    quat_to_rot(st->qn, st->Rq);
    for (int c = 0; c < 3; c++) st->s[c] = exp(scale[4 * i + c]);
    double M[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) M[3 * r + c] = st->Rq[3 * r + c] * st->s[c];
    double MT[9];
    mat3_T(M, MT);
    mat3_mul(M, MT, st->Sig);
    double RT[9], tmp[9];
    mat3_T(k->R, RT);
    mat3_mul(k->R, st->Sig, tmp);
    mat3_mul(tmp, RT, st->Sc);

    double limx = 1.3 * (k->W * 0.5) / k->fx, limy = 1.3 * (k->H * 0.5) / k->fy;
    double xz = x / z, yz = y / z;
    if (fabs(fabs(xz) - limx) < g->m_geo * limx) a |= 2;
    if (fabs(fabs(yz) - limy) < g->m_geo * limy) a |= 2;
    st->clamp_x = xz < -limx || xz > limx;
    st->clamp_y = yz < -limy || yz > limy;
    double cxz = xz < -limx ? -limx : (xz > limx ? limx : xz);
    double cyz = yz < -limy ? -limy : (yz > limy ? limy : yz);
    double* J = st->J;
    J[0] = k->fx / z; J[1] = 0; J[2] = -k->fx * cxz / z;
    J[3] = 0; J[4] = k->fy / z; J[5] = -k->fy * cyz / z;
    /* S2 = J Sc J^T + dil I */
    double JS[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            JS[3 * r + c] = J[3 * r] * st->Sc[c] + J[3 * r + 1] * st->Sc[3 + c] + J[3 * r + 2] * st->Sc[6 + c];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++)
            st->S2[2 * r + c] = JS[3 * r] * J[3 * c] + JS[3 * r + 1] * J[3 * c + 1] + JS[3 * r + 2] * J[3 * c + 2];
    /* filter factor: rho = det(Sigma2D) / det(Sigma2D + dil I), before the dilation */
    double det0 = st->S2[0] * st->S2[3] - st->S2[1] * st->S2[1];
    double a0 = st->S2[0], c0 = st->S2[3];
    st->S2[0] += g->dil;
    st->S2[3] += g->dil;
    double A = st->S2[0], Bc = st->S2[1], C = st->S2[3];
    st->det = A * C - Bc * Bc;
    if (fabs(st->det) < g->m_geo * A * C) a |= 1;
    st->rho = 1.0; st->fmip = 1.0; st->rho_floor = 0;
    if (g->mip) {
        st->rho = det0 / st->det;
        /* an FP32 det(Sigma2D) of a very thin splat (det0 << a0 c0) may lose most digits */
        if (fabs(det0) < 1e-4 * a0 * c0 || fabs(st->rho - 1e-6) < g->m_geo * 1e-6) a |= 1;
        st->rho_floor = !(st->rho > 1e-6);
        st->fmip = sqrt(st->rho_floor ? 1e-6 : st->rho);
    }
    if (amb) amb[i] = a;
    if (!(st->det > 0)) return;
    double u = k->fx * x / z + k->cx, v = k->fy * y / z + k->cy;
    double mid = 0.5 * (A + C);
    double lam = mid + sqrt(fmax(0.1, mid * mid - st->det));
    double q3 = 3.0 * sqrt(lam);
    /* a radius near an integer may round to r or r+1: an edge then moves by 1 px */
    double r_slack = dist_to_int(q3) < g->m_geo * fmax(1.0, q3) ? 1.0 : 0.0;
    double r = ceil(q3);
    int T = g->tile;
    int tx = (k->W + T - 1) / T, ty = (k->H + T - 1) / T;
    double e[4] = {(u - r) / T, (v - r) / T, (u + r + T - 1) / T, (v + r + T - 1) / T};
    double lim[4] = {tx, ty, tx, ty};
    /* opacity-aware bounds (alpha_rect): edges of the box where alpha reaches alpha_min */
    double o_eff = st->fmip / (1.0 + exp(-logit));
    int use_a = g->alpha_rect != 0, a_empty = 0;
    double ea[4] = {0, 0, 0, 0};
    if (use_a) {
        /* bit 64: an opacity within the margin of alpha_min may list the item or not in FP32 */
        if (fabs(o_eff - g->a_min) < g->m_alpha * g->a_min) a |= 64;
        if (!(o_eff >= g->a_min)) {
            a_empty = 1;
        } else {
            double ta = 2.0 * log(o_eff / g->a_min);
            double hx = sqrt(ta * A), hy = sqrt(ta * C);
            ea[0] = (u - hx) / T; ea[1] = (v - hy) / T; ea[2] = (u + hx) / T + 1.0; ea[3] = (v + hy) / T + 1.0;
        }
    }
    /* an edge near a tile boundary inside the grid may round either way in fp32;
     * bits 4, 8, 16, 32 flag edges x0, y0, x1, y1. side (optional) says which
     * way the other rounding goes: bit c set when the edge lies at or above the
     * boundary (floor gives the boundary; the other rounding is one less), bit
     * 4 + c when a radius near an integer may move the edge either way. */
    uint8_t sd = 0;
    int rc[4], ra[4];
    for (int c = 0; c < 4; c++) {
        double f = floor(e[c]);
        if (f < 0) f = 0;
        if (f > lim[c]) f = lim[c];
        rc[c] = (int)f;
        double fa = floor(ea[c]);
        if (fa < 0) fa = 0;
        if (fa > lim[c]) fa = lim[c];
        ra[c] = (int)fa;
    }
    for (int c = 0; c < 4; c++) {
        /* the binding edge of the two (the larger lower bound, the smaller upper bound; both when equal) */
        /* an opacity below alpha_min lists the item nowhere whatever its edges (bit 64 flags it near) */
        int bind3 = !(use_a && a_empty), binda = 0;
        if (use_a && !a_empty) {
            binda = c < 2 ? ra[c] >= rc[c] : ra[c] <= rc[c];
            bind3 = c < 2 ? rc[c] >= ra[c] : rc[c] <= ra[c];
        }
        double kk = nearbyint(e[c]);
        if (bind3 && kk >= 1 && kk <= lim[c] && dist_to_int(e[c]) * T < g->m_rect + r_slack) {
            a |= (uint8_t)(4 << c);
            if (e[c] >= kk) sd |= (uint8_t)(1 << c);
            if (r_slack > 0) sd |= (uint8_t)(16 << c);
        } else if (binda) {
            double ka = nearbyint(ea[c]);
            if (ka >= 1 && ka <= lim[c] && dist_to_int(ea[c]) * T < g->m_rect) {
                a |= (uint8_t)(4 << c);
                if (ea[c] >= ka) sd |= (uint8_t)(1 << c);
            }
        }
    }
    if (side) side[i] = sd;
    if (use_a) {
        if (a_empty) {
            rc[2] = rc[0];  /* the opacity never reaches alpha_min: listed nowhere */
        } else {
            if (ra[0] > rc[0]) rc[0] = ra[0];
            if (ra[1] > rc[1]) rc[1] = ra[1];
            if (ra[2] < rc[2]) rc[2] = ra[2];
            if (ra[3] < rc[3]) rc[3] = ra[3];
            if (rc[2] < rc[0]) rc[2] = rc[0];
            if (rc[3] < rc[1]) rc[3] = rc[1];
        }
    }
    if (amb) amb[i] = a;
    if (!isfinite(u) || !isfinite(v)) return;
    /* An empty rect lists the item in no tile, so it stays culled; its
     * projected values and clamped rect are written all the same, because a
     * rect edge within the margin may make it one tile wide in FP32. */
    int empty = (rc[2] - rc[0]) * (rc[3] - rc[1]) == 0;

    /* colour from SH in the direction camera centre -> mean */
    double cpos[3];
    for (int c = 0; c < 3; c++) cpos[c] = -(RT[3 * c] * k->t[0] + RT[3 * c + 1] * k->t[1] + RT[3 * c + 2] * k->t[2]);
    for (int c = 0; c < 3; c++) st->dir[c] = mu[c] - cpos[c];
    st->dlen = sqrt(st->dir[0] * st->dir[0] + st->dir[1] * st->dir[1] + st->dir[2] * st->dir[2]);
    for (int c = 0; c < 3; c++) st->d[c] = st->dir[c] / st->dlen;
    or_sh_basis(g->sh_degree, st->d, st->Y, st->dY);
    int ncoef = (g->sh_degree + 1) * (g->sh_degree + 1);
    double col[3];
    uint8_t cm = 0;
    for (int ch = 0; ch < 3; ch++) {
        double s = 0.5;
        for (int kk = 0; kk < ncoef; kk++) s += st->Y[kk] * sh[48 * i + 3 * kk + ch];
        st->raw[ch] = s;
        if (fabs(s) < g->m_geo) a |= 2;
        col[ch] = s > 0 ? s : 0;
        if (s < 0) cm |= (uint8_t)(1 << ch);
    }
    double o = 1.0 / (1.0 + exp(-logit));
    st->o = o;
    o *= st->fmip;
    if (!isfinite(st->raw[0]) || !isfinite(st->raw[1]) || !isfinite(st->raw[2]) || !isfinite(o)) return;

    st->culled = empty;
    mean2d[2 * i] = u; mean2d[2 * i + 1] = v;
    conic[3 * i] = C / st->det; conic[3 * i + 1] = -Bc / st->det; conic[3 * i + 2] = A / st->det;
    opac[i] = o;
    for (int ch = 0; ch < 3; ch++) rgb[3 * i + ch] = col[ch];
    for (int c = 0; c < 4; c++) rect[4 * i + c] = rc[c];
    if (clampm) clampm[i] = cm;
    if (amb) amb[i] = a;
}

/* Returns the number of visible Gaussians. Outputs are per Gaussian; culled ones
 * get n_tiles = 0 (an all-zero rect when culled before the rect, else the
 * empty rect as computed). depth_key is the depth rounded to fp32. side
 * (optional) as in project_one. */
int64_t or_project(int64_t n, const double* mean_opa, const double* scale, const double* quat, const double* sh,
                   const double* cam, const double* cfg, double* mean2d, double* conic, double* opac,
                   double* rgb, double* depth, float* depth_key, int32_t* rect, int32_t* n_tiles,
                   uint8_t* clampm, uint8_t* amb, uint8_t* side) {
    Cam k = read_cam(cam);
    Cfg g = read_cfg(cfg);
    int64_t vis = 0;
#pragma omp parallel for schedule(static) reduction(+ : vis)
    for (int64_t i = 0; i < n; i++) {
        ProjState st;
        mean2d[2 * i] = mean2d[2 * i + 1] = 0;
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
        opac[i] = 0;
        rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0;
        if (clampm) clampm[i] = 0;
        if (side) side[i] = 0;
        project_one(i, mean_opa, scale, quat, sh, &k, &g, &st, mean2d, conic, opac, rgb, depth, rect, clampm, amb,
                    side);
        depth_key[i] = (float)depth[i];
        n_tiles[i] = (rect[4 * i + 2] - rect[4 * i]) * (rect[4 * i + 3] - rect[4 * i + 1]);
        vis += !st.culled;
    }
    return vis;
}

/* ---------------------------------------------------------------------------
 * Per-tile lists: every (tile, Gaussian) pair whose rect holds the tile, each
 * tile's list ordered by (fp32 depth bits, Gaussian id).
 * ------------------------------------------------------------------------- */
typedef struct { uint32_t key; int32_t id; } KeyId;

static int cmp_keyid(const void* pa, const void* pb) {
    const KeyId* a = (const KeyId*)pa;
    const KeyId* b = (const KeyId*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* tile_start has tiles_x*tiles_y+1 entries. Returns the total pair count; fills
 * ids only if it fits in capacity. */
int64_t or_tile_lists(int64_t n, const int32_t* rect, const float* depth_key, int tiles_x, int tiles_y,
                      int64_t* tile_start, int32_t* ids, int64_t capacity) {
    int64_t nt = (int64_t)tiles_x * tiles_y;
    for (int64_t t = 0; t <= nt; t++) tile_start[t] = 0;
    for (int64_t i = 0; i < n; i++)
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ty++)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; tx++) tile_start[(int64_t)ty * tiles_x + tx + 1]++;
    for (int64_t t = 0; t < nt; t++) tile_start[t + 1] += tile_start[t];
    int64_t total = tile_start[nt];
    if (total > capacity) return total;
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (nt > 0 ? nt : 1));
    for (int64_t t = 0; t < nt; t++) fill[t] = tile_start[t];
    for (int64_t i = 0; i < n; i++)
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ty++)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; tx++) ids[fill[(int64_t)ty * tiles_x + tx]++] = (int32_t)i;
    free(fill);
#pragma omp parallel
    {
        KeyId* buf = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nt; t++) {
            int64_t b = tile_start[t], e = tile_start[t + 1];
            if (e - b > cap) { cap = e - b; buf = (KeyId*)realloc(buf, sizeof(KeyId) * cap); }
            for (int64_t j = b; j < e; j++) {
                uint32_t bits;
                memcpy(&bits, &depth_key[ids[j]], 4);
                buf[j - b].key = bits;
                buf[j - b].id = ids[j];
            }
            qsort(buf, (size_t)(e - b), sizeof(KeyId), cmp_keyid);
            for (int64_t j = b; j < e; j++) ids[j] = buf[j - b].id;
        }
        free(buf);
    }
    return total;
}

/* ---------------------------------------------------------------------------
 * Front-to-back alpha compositing, per pixel.
 * ------------------------------------------------------------------------- */
typedef struct {
    double alpha, T, g, og;  /* alpha, transmittance before it, exp(power), o*exp(power) */
    int32_t id;
    int clamped;
    int64_t j;               /* position in the pixel's list */
    double dpow;             /* uncertainty of the FP32 exponent (margins only) */
} Contrib;

/* Decisions of the compositing loop that can be recorded when within their
 * margin, and forced to the other branch (the tolerance bounds use this). */
enum { FL_POWER = 1, FL_CLAMP = 2, FL_AMIN = 3, FL_TMIN = 4, FL_DEPTH = 5 };
typedef struct {
    int64_t j, j2; /* list position of the decision; FL_DEPTH: also the earlier Gaussian of the near-tie */
    int kind;
} Flag;

/* Walks the pixel's list; records composited Gaussians into rec (if non-NULL).
 * Returns the number composited; sets *n_contrib, *T_out, color. A decision
 * within the margins sets *amb and, when amb_g is given, flags the Gaussian(s)
 * it concerns; when flags is given the decision is also appended there (at
 * most max_flags, counted in *n_flags). flip (may be NULL) names one decision
 * (list position and kind, not FL_DEPTH) that is forced to the other branch. */
static int composite_pixel(const Cfg* g, double px, double py, const int32_t* ids, int64_t len,
                           const double* mean2d, const double* conic, const double* opac, const double* rgb,
                           const double* depth, double* color, double* T_out, int32_t* n_contrib, uint8_t* amb,
                           Contrib* rec, uint8_t* amb_g, const Flag* flip, Flag* flags, int max_flags,
                           int* n_flags) {
    double T = 1.0, C[3] = {0, 0, 0};
    int nrec = 0;
    int32_t last = 0;
    double z_prev = -1.0;
    int32_t id_prev = -1;
    int64_t j_prev = -1;
    /* Relative uncertainty of the FP32 path's T, grown by each composited
     * Gaussian's alpha uncertainty and one rounding per step (margins only:
     * the arithmetic above is unaffected). */
    double T_unc = 0.0;
#define FLAG_G(x)                          \
    do {                                   \
        *amb = 1;                          \
        if (amb_g) {                       \
            _Pragma("omp atomic write")    \
            amb_g[x] = 1;                  \
        }                                  \
    } while (0)
#define RECORD(jj, kk, j2_)                                                   \
    do {                                                                      \
        if (flags && *n_flags < max_flags) {                                  \
            flags[*n_flags].j = (jj); flags[*n_flags].j2 = (j2_);             \
            flags[*n_flags].kind = (kk); (*n_flags)++;                        \
        }                                                                     \
    } while (0)
#define FORCED(jj, kk) (flip && flip->j == (jj) && flip->kind == (kk))
    if (n_flags) *n_flags = 0;
    for (int64_t j = 0; j < len; j++) {
        int32_t id = ids[j];
        double dx = px - mean2d[2 * id], dy = py - mean2d[2 * id + 1];
        double a = conic[3 * id], b = conic[3 * id + 1], c = conic[3 * id + 2];
        double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        /* Uncertainty of the FP32 exponent: the splat centre is held in FP32
         * (a few ulps of its coordinates), times the exponent's gradient, plus
         * the conic's relative rounding and the hardware exp2. At 1080p an ulp
         * of a coordinate is up to 1.2e-4 px, which for the narrowest splats
         * moves alpha by ~1e-3 relative. */
        double ulp = 4.0 * ldexp(fmax(1.0, fmax(fabs(mean2d[2 * id]), fabs(mean2d[2 * id + 1]))), -24);
        double grad = fabs(a * dx + b * dy) + fabs(c * dy + b * dx);
        double dpow = grad * ulp + 1e-5 * fabs(power) + ldexp(1.0, -21);
        if (fabs(power) < dpow) { FLAG_G(id); RECORD(j, FL_POWER, -1); }
        if ((power > 0) != FORCED(j, FL_POWER)) continue;
        double G = exp(power);
        double og = opac[id] * G;
        if (fabs(og - g->a_max) < (g->m_alpha + dpow) * g->a_max) { FLAG_G(id); RECORD(j, FL_CLAMP, -1); }
        int clamped = !(og < g->a_max);
        if (FORCED(j, FL_CLAMP)) clamped = !clamped;
        double alpha = clamped ? g->a_max : og;
        if (fabs(alpha - g->a_min) < (g->m_alpha + dpow) * g->a_min) { FLAG_G(id); RECORD(j, FL_AMIN, -1); }
        if ((alpha < g->a_min) != FORCED(j, FL_AMIN)) continue;
        double testT = T * (1.0 - alpha);
        double t_unc = T_unc + alpha / (1.0 - alpha) * dpow + ldexp(1.0, -22);
        if (fabs(testT - g->t_min) < (g->m_T + t_unc) * g->t_min) { FLAG_G(id); RECORD(j, FL_TMIN, -1); }
        if ((testT < g->t_min) != FORCED(j, FL_TMIN)) break;
        T_unc = t_unc;
        if (depth) {
            if (z_prev >= 0 && fabs(depth[id] - z_prev) <= g->m_depth * fabs(depth[id])) {
                FLAG_G(id);
                FLAG_G(id_prev);
                RECORD(j, FL_DEPTH, j_prev);
            }
            z_prev = depth[id];
            id_prev = id;
            j_prev = j;
        }
        for (int ch = 0; ch < 3; ch++) C[ch] += alpha * T * rgb[3 * id + ch];
        if (rec) {
            rec[nrec].alpha = alpha; rec[nrec].T = T; rec[nrec].g = G; rec[nrec].og = og;
            rec[nrec].id = id; rec[nrec].clamped = clamped; rec[nrec].j = j; rec[nrec].dpow = dpow;
        }
        nrec++;
        T = testT;
        last = (int32_t)(j + 1);
    }
    for (int ch = 0; ch < 3; ch++) color[ch] = C[ch] + T * g->bg[ch];
    *T_out = T;
    *n_contrib = last;
    return nrec;
#undef FORCED
#undef RECORD
#undef FLAG_G
}

void or_render_fwd(const double* cam, const double* cfg, const int64_t* tile_start, const int32_t* ids,
                   const double* mean2d, const double* conic, const double* opac, const double* rgb,
                   const double* depth, double* color, double* t_final, int32_t* n_contrib, uint8_t* amb_px,
                   uint8_t* amb_g, int32_t* n_comp) {
    Cam k = read_cam(cam);
    Cfg g = read_cfg(cfg);
    int T = g.tile, tx = (k.W + T - 1) / T;
    int64_t HW = (int64_t)k.W * k.H;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t pix = 0; pix < HW; pix++) {
        int x = (int)(pix % k.W), y = (int)(pix / k.W);
        int64_t t = (int64_t)(y / T) * tx + x / T;
        double col[3], Tf;
        int32_t nc;
        uint8_t a = 0;
        int nr = composite_pixel(&g, x + 0.5, y + 0.5, ids + tile_start[t], tile_start[t + 1] - tile_start[t],
                                 mean2d, conic, opac, rgb, depth, col, &Tf, &nc, &a, NULL, amb_g, NULL, NULL, 0,
                                 NULL);
        if (n_comp) n_comp[pix] = nr;
        for (int ch = 0; ch < 3; ch++) color[ch * HW + pix] = col[ch];
        t_final[pix] = Tf;
        n_contrib[pix] = nc;
        if (amb_px) amb_px[pix] = a;
    }
}

/* Adjoint of one pixel's compositing. rec[0..nr) are the pixel's composited
 * Gaussians in front-to-back order (from composite_pixel, final transmittance
 * Tf); with C = sum_i alpha_i T_i c_i + T_N bg,
 *   dC/dc_i     = alpha_i T_i
 *   dC/dalpha_i = T_i c_i - (sum_{j>i} alpha_j T_j c_j + T_N bg) / (1 - alpha_i),
 * then alpha = min(a_max, o g), g = exp(power),
 * power = -(a dx^2 + c dy^2)/2 - b dx dy, d = pixel - mean2d.
 * out[9 r + q] = this pixel's share of dL/d(u, v, conic a, b, c, opacity,
 * r, g, b) of rec[r] for the colour gradient gC; the first six are 0 where
 * alpha is clamped. */
static void pixel_contribs(const Cfg* g, double px, double py, const Contrib* rec, int nr, double Tf,
                           const double* mean2d, const double* conic, const double* rgb, const double* gC,
                           double* out) {
    double total[3] = {0, 0, 0};
    for (int r = 0; r < nr; r++)
        for (int ch = 0; ch < 3; ch++) total[ch] += rec[r].alpha * rec[r].T * rgb[3 * rec[r].id + ch];
    double prefix[3] = {0, 0, 0};
    for (int r = 0; r < nr; r++) {
        const Contrib* c = &rec[r];
        int32_t id = c->id;
        double* o = out + 9 * r;
        double dalpha = 0;
        for (int ch = 0; ch < 3; ch++) {
            double ci = rgb[3 * id + ch];
            prefix[ch] += c->alpha * c->T * ci;
            double after = total[ch] - prefix[ch];
            o[6 + ch] = c->alpha * c->T * gC[ch];
            dalpha += gC[ch] * (c->T * ci - (after + Tf * g->bg[ch]) / (1.0 - c->alpha));
        }
        for (int q = 0; q < 6; q++) o[q] = 0;
        if (!c->clamped) {
            double dpower = dalpha * c->og;
            double dx = px - mean2d[2 * id], dy = py - mean2d[2 * id + 1];
            double ca = conic[3 * id], cb = conic[3 * id + 1], cc = conic[3 * id + 2];
            /* dpower/du = a dx + b dy, dpower/dv = b dx + c dy (d = pixel - mean) */
            o[0] = dpower * (ca * dx + cb * dy);
            o[1] = dpower * (cb * dx + cc * dy);
            o[2] = dpower * (-0.5 * dx * dx);
            o[3] = dpower * (-dx * dy);
            o[4] = dpower * (-0.5 * dy * dy);
            o[5] = dalpha * c->g;
        }
    }
}

/* Adjoint of the compositing, one view: the per-pixel adjoint above summed over
 * the pixels of every tile. g2d[9*i] = dL/d(u, v, conic a, b, c, opacity,
 * r, g, b) of item i. amb_g2d (optional, same shape): the sum of
 * |contribution| coming from pixels flagged ambiguous (by this pass, or in
 * amb_in [H*W] when given). */
void or_render_bwd(const double* cam, const double* cfg, const int64_t* tile_start, const int32_t* ids,
                   const double* mean2d, const double* conic, const double* opac, const double* rgb,
                   const double* depth, const double* dL_dcolor, int64_t n, double* g2d, double* amb_g2d,
                   const uint8_t* amb_in) {
    Cam k = read_cam(cam);
    Cfg g = read_cfg(cfg);
    int T = g.tile, tx = (k.W + T - 1) / T, ty = (k.H + T - 1) / T;
    int64_t HW = (int64_t)k.W * k.H, nt = (int64_t)tx * ty;
    int64_t P = tile_start[nt];
    /* one partial per list entry so tiles can run in parallel; summed in list order below */
    double* part = (double*)calloc((size_t)(P > 0 ? P : 1) * 9, sizeof(double));
    double* part_amb = (double*)calloc((size_t)(P > 0 ? P : 1) * 9, sizeof(double));
#pragma omp parallel
    {
        int64_t cap = 0;
        Contrib* rec = NULL;
        double* cb = NULL;
#pragma omp for schedule(dynamic, 8)
        for (int64_t t = 0; t < nt; t++) {
            int64_t b0 = tile_start[t], len = tile_start[t + 1] - b0;
            if (len > cap) {
                cap = len;
                rec = (Contrib*)realloc(rec, sizeof(Contrib) * cap);
                cb = (double*)realloc(cb, sizeof(double) * 9 * cap);
            }
            int x0 = (int)(t % tx) * T, y0 = (int)(t / tx) * T;
            for (int y = y0; y < y0 + T && y < k.H; y++)
                for (int x = x0; x < x0 + T && x < k.W; x++) {
                    int64_t pix = (int64_t)y * k.W + x;
                    double col[3], Tf, px = x + 0.5, py = y + 0.5;
                    int32_t nc;
                    uint8_t a = 0;
                    int nr = composite_pixel(&g, px, py, ids + b0, len, mean2d, conic, opac, rgb, depth, col, &Tf, &nc,
                                             &a, rec, NULL, NULL, NULL, 0, NULL);
                    if (amb_in && amb_in[pix]) a = 1;
                    double gC[3] = {dL_dcolor[pix], dL_dcolor[HW + pix], dL_dcolor[2 * HW + pix]};
                    pixel_contribs(&g, px, py, rec, nr, Tf, mean2d, conic, rgb, gC, cb);
                    for (int r = 0; r < nr; r++) {
                        double* pp = part + 9 * (b0 + rec[r].j);
                        const double* o = cb + 9 * r;
                        double before[9];
                        for (int q = 0; q < 9; q++) before[q] = pp[q];
                        for (int q = 6; q < 9; q++) pp[q] += o[q];
                        if (!rec[r].clamped)
                            for (int q = 0; q < 6; q++) pp[q] += o[q];
                        if (a)
                            for (int q = 0; q < 9; q++) part_amb[9 * (b0 + rec[r].j) + q] += fabs(pp[q] - before[q]);
                    }
                }
        }
        free(rec);
        free(cb);
    }
    for (int64_t i = 0; i < 9 * n; i++) g2d[i] = 0;
    if (amb_g2d)
        for (int64_t i = 0; i < 9 * n; i++) amb_g2d[i] = 0;
    for (int64_t j = 0; j < P; j++)
        for (int c = 0; c < 9; c++) {
            g2d[9 * (int64_t)ids[j] + c] += part[9 * j + c];
            if (amb_g2d) amb_g2d[9 * (int64_t)ids[j] + c] += part_amb[9 * j + c];
        }
    free(part);
    free(part_amb);
}

/* ---------------------------------------------------------------------------
 * Adjoint of the projection, one view: from g2d (per Gaussian, as written by
 * or_render_bwd) to the parameter gradients and the camera pose gradient.
 * Outputs are overwritten (culled Gaussians get zeros). g_pose[6] = dL/d(rho, phi)
 * for T_cw <- exp(xi^) T_cw.
 * ------------------------------------------------------------------------- */
static void sym2_from(double a, double b, double c, double* M) { M[0] = a; M[1] = b; M[2] = b; M[3] = c; }

/* Adjoint of the projection for one visible item (st from project_one): from
 * its 2D adjoint G[9] to its parameter gradients, overwritten in gm[3],
 * *glogit, gls[3], gq4[4], gsh[48], and its camera-pose contribution, added to
 * pose[6]. Linear in G. */
static void project_bwd_item(const ProjState* pst, const double* G, const double* shrow, const Cam* kp,
                         const Cfg* gp_, double* gm, double* glogit, double* gls, double* gq4, double* gsh,
                         double* pose) {
    const ProjState st = *pst;
    const Cam k = *kp;
    const Cfg g = *gp_;
    int ncoef = (g.sh_degree + 1) * (g.sh_degree + 1);
    for (int c = 0; c < 3; c++) gm[c] = 0, gls[c] = 0;
    for (int c = 0; c < 4; c++) gq4[c] = 0;
    for (int c = 0; c < 48; c++) gsh[c] = 0;
    *glogit = 0;
    double x = st.p[0], y = st.p[1], z = st.p[2];

    /* opacity o f, o = sigmoid(logit), f = sqrt(rho) with the filter (else 1) */
    *glogit = G[5] * st.fmip * st.o * (1 - st.o);
    double g_rho = (g.mip && !st.rho_floor) ? G[5] * st.o / (2.0 * st.fmip) : 0.0;

    /* colour: rgb = max(SH(d) + 0.5, 0) */
    double graw[3];
    for (int ch = 0; ch < 3; ch++) graw[ch] = st.raw[ch] > 0 ? G[6 + ch] : 0;
    double gd[3] = {0, 0, 0};
    for (int kk = 0; kk < ncoef; kk++)
        for (int ch = 0; ch < 3; ch++) {
            double shv = shrow[3 * kk + ch];
            gsh[3 * kk + ch] = graw[ch] * st.Y[kk];
            for (int c = 0; c < 3; c++) gd[c] += graw[ch] * shv * st.dY[3 * kk + c];
        }
    /* d = dir/|dir|: dL/ddir = (gd - d (d.gd)) / |dir| */
    double dd = gd[0] * st.d[0] + gd[1] * st.d[1] + gd[2] * st.d[2];
    double gdir[3];
    for (int c = 0; c < 3; c++) gdir[c] = (gd[c] - st.d[c] * dd) / st.dlen;
    for (int c = 0; c < 3; c++) gm[c] += gdir[c];
    if (g.pose_through_sh) {
        /* dir = mu - centre, centre = -R^T t; left perturbation moves the centre by -R^T rho */
        for (int r = 0; r < 3; r++)
            pose[r] += k.R[3 * r] * gdir[0] + k.R[3 * r + 1] * gdir[1] + k.R[3 * r + 2] * gdir[2];
    }

    /* conic = S2^-1: dL/dS2 = -Q dL/dQ Q with the full symmetric dL/dQ */
    double Q[4], GQ[4], GS[4], t4[4];
    sym2_from(st.S2[3] / st.det, -st.S2[1] / st.det, st.S2[0] / st.det, Q);
    sym2_from(G[2], 0.5 * G[3], G[4], GQ);
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) t4[2 * r + c] = Q[2 * r] * GQ[c] + Q[2 * r + 1] * GQ[2 + c];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) GS[2 * r + c] = -(t4[2 * r] * Q[c] + t4[2 * r + 1] * Q[2 + c]);
    if (g_rho != 0.0) {
        /* rho = ((A - dil)(C - dil) - B^2) / (A C - B^2) with S2 = [[A, B], [B, C]] */
        double A = st.S2[0], B = st.S2[1], C = st.S2[3], rho = st.rho;
        GS[0] += g_rho * ((C - g.dil) - rho * C) / st.det;
        GS[3] += g_rho * ((A - g.dil) - rho * A) / st.det;
        GS[1] += -g_rho * B * (1.0 - rho) / st.det; /* half of d rho / dB on each symmetric entry */
        GS[2] += -g_rho * B * (1.0 - rho) / st.det;
    }

    /* S2 = J Sc J^T + dil I: dL/dSc = J^T GS J, dL/dJ = 2 GS J Sc */
    const double* J = st.J;
    double GSc[9], GJ[6], JSc[6];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double s = 0;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) s += J[3 * a + r] * GS[2 * a + b] * J[3 * b + c];
            GSc[3 * r + c] = s;
        }
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            JSc[3 * r + c] = J[3 * r] * st.Sc[c] + J[3 * r + 1] * st.Sc[3 + c] + J[3 * r + 2] * st.Sc[6 + c];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) GJ[3 * r + c] = 2 * (GS[2 * r] * JSc[c] + GS[2 * r + 1] * JSc[3 + c]);

    /* mean2d and J as functions of p = (x, y, z) */
    double gp[3] = {0, 0, 0};
    gp[0] += G[0] * k.fx / z;
    gp[2] += -G[0] * k.fx * x / (z * z);
    gp[1] += G[1] * k.fy / z;
    gp[2] += -G[1] * k.fy * y / (z * z);
    gp[2] += GJ[0] * (-k.fx / (z * z)) + GJ[4] * (-k.fy / (z * z));
    if (st.clamp_x) {
        double c = x / z < 0 ? -1.3 * (k.W * 0.5) / k.fx : 1.3 * (k.W * 0.5) / k.fx;
        gp[2] += GJ[2] * (k.fx * c / (z * z));
    } else {
        gp[0] += GJ[2] * (-k.fx / (z * z));
        gp[2] += GJ[2] * (2 * k.fx * x / (z * z * z));
    }
    if (st.clamp_y) {
        double c = y / z < 0 ? -1.3 * (k.H * 0.5) / k.fy : 1.3 * (k.H * 0.5) / k.fy;
        gp[2] += GJ[5] * (k.fy * c / (z * z));
    } else {
        gp[1] += GJ[5] * (-k.fy / (z * z));
        gp[2] += GJ[5] * (2 * k.fy * y / (z * z * z));
    }

    /* Sc = R Sig R^T: dL/dSig = R^T GSc R */
    double RT[9], t9[9], GSig[9];
    mat3_T(k.R, RT);
    mat3_mul(RT, GSc, t9);
    mat3_mul(t9, k.R, GSig);
    /* Sig = M M^T, M = Rq diag(s): dL/dM = 2 GSig M */
    double M[9], GM[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) M[3 * r + c] = st.Rq[3 * r + c] * st.s[c];
    mat3_mul(GSig, M, GM);
    for (int c = 0; c < 9; c++) GM[c] *= 2;
    double GRq[9];
    for (int c = 0; c < 3; c++) {
        double gs = 0;
        for (int r = 0; r < 3; r++) {
            gs += GM[3 * r + c] * st.Rq[3 * r + c];
            GRq[3 * r + c] = GM[3 * r + c] * st.s[c];
        }
        gls[c] = gs * st.s[c];
    }
    /* rotation matrix of the normalised quaternion */
    double w = st.qn[0], qx = st.qn[1], qy = st.qn[2], qz = st.qn[3];
    double gq[4];
    gq[0] = 2 * (-qz * GRq[1] + qy * GRq[2] + qz * GRq[3] - qx * GRq[5] - qy * GRq[6] + qx * GRq[7]);
    gq[1] = 2 * (qy * GRq[1] + qz * GRq[2] + qy * GRq[3] - 2 * qx * GRq[4] - w * GRq[5] + qz * GRq[6] + w * GRq[7] - 2 * qx * GRq[8]);
    gq[2] = 2 * (-2 * qy * GRq[0] + qx * GRq[1] + w * GRq[2] + qx * GRq[3] + qz * GRq[5] - w * GRq[6] + qz * GRq[7] - 2 * qy * GRq[8]);
    gq[3] = 2 * (-2 * qz * GRq[0] - w * GRq[1] + qx * GRq[2] + w * GRq[3] - 2 * qz * GRq[4] + qy * GRq[5] + qx * GRq[6] + qy * GRq[7]);
    double qd = gq[0] * st.qn[0] + gq[1] * st.qn[1] + gq[2] * st.qn[2] + gq[3] * st.qn[3];
    for (int c = 0; c < 4; c++) gq4[c] = (gq[c] - st.qn[c] * qd) / st.qlen;

    /* p = R mu + t */
    for (int c = 0; c < 3; c++) gm[c] += RT[3 * c] * gp[0] + RT[3 * c + 1] * gp[1] + RT[3 * c + 2] * gp[2];

    /* pose, left perturbation: dp = rho + phi x p, dSc = phi^ Sc - Sc phi^ */
    pose[0] += gp[0]; pose[1] += gp[1]; pose[2] += gp[2];
    pose[3] += st.p[1] * gp[2] - st.p[2] * gp[1];
    pose[4] += st.p[2] * gp[0] - st.p[0] * gp[2];
    pose[5] += st.p[0] * gp[1] - st.p[1] * gp[0];
    double A1[9], A2[9], Mx[9];
    mat3_mul(st.Sc, GSc, A1);
    mat3_mul(GSc, st.Sc, A2);
    for (int c = 0; c < 9; c++) Mx[c] = A1[c] - A2[c];
    pose[3] += Mx[5] - Mx[7];
    pose[4] += Mx[6] - Mx[2];
    pose[5] += Mx[1] - Mx[3];
}

void or_project_bwd(int64_t n, const double* mean_opa, const double* scale, const double* quat, const double* sh,
                    const double* cam, const double* cfg, const double* g2d, double* g_mean, double* g_logit,
                    double* g_logscale, double* g_quat, double* g_sh, double* g_pose) {
    Cam k = read_cam(cam);
    Cfg g = read_cfg(cfg);
    double pose[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
        ProjState st;
        double m2[2], cn[3], op, col[3], dep;
        int32_t rc[4];
        for (int c = 0; c < 3; c++) g_mean[3 * i + c] = 0, g_logscale[3 * i + c] = 0;
        for (int c = 0; c < 4; c++) g_quat[4 * i + c] = 0;
        for (int c = 0; c < 48; c++) g_sh[48 * i + c] = 0;
        g_logit[i] = 0;
        /* project_one indexes its outputs by i; point it at local storage */
        project_one(0, mean_opa + 4 * i, scale + 4 * i, quat + 4 * i, sh + 48 * i, &k, &g, &st, m2, cn, &op, col,
                    &dep, rc, NULL, NULL, NULL);
        if (st.culled) continue;
        project_bwd_item(&st, g2d + 9 * i, sh + 48 * i, &k, &g, g_mean + 3 * i, g_logit + i, g_logscale + 3 * i,
                         g_quat + 4 * i, g_sh + 48 * i, pose);
    }
    for (int c = 0; c < 6; c++) g_pose[c] = pose[c];
}

/* Bounds carried through the projection adjoint. b2d[9 i + c] >= 0 bounds how
 * far the 2D adjoint component c of item i may be from the value the oracle
 * computes. The adjoint is linear in the 2D adjoint, so the most a parameter
 * gradient can move is sum_c |d param / d g2d_c| b2d_c, and the most the
 * view's pose gradient can move is the sum of that over the items; each
 * Jacobian column is the item adjoint of a unit vector. Outputs (overwritten)
 * have the shapes of or_project_bwd's. With g2d given (may be NULL),
 * pose_absum[6] receives sum_i |pose contribution of item i| under that
 * adjoint: the scale of the rounding error of summing the items in any order. */
void or_project_bwd_abs(int64_t n, const double* mean_opa, const double* scale, const double* quat,
                        const double* sh, const double* cam, const double* cfg, const double* b2d,
                        const double* g2d, double* b_mean, double* b_logit, double* b_logscale, double* b_quat,
                        double* b_sh, double* b_pose, double* pose_absum) {
    Cam k = read_cam(cam);
    Cfg g = read_cfg(cfg);
    double* item_pose = (double*)calloc((size_t)(n > 0 ? n : 1) * 12, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        ProjState st;
        double m2[2], cn[3], op, col[3], dep;
        int32_t rc[4];
        double gm[3], gl, gls[3], gq[4], gsh[48];
        for (int c = 0; c < 3; c++) b_mean[3 * i + c] = 0, b_logscale[3 * i + c] = 0;
        for (int c = 0; c < 4; c++) b_quat[4 * i + c] = 0;
        for (int c = 0; c < 48; c++) b_sh[48 * i + c] = 0;
        b_logit[i] = 0;
        project_one(0, mean_opa + 4 * i, scale + 4 * i, quat + 4 * i, sh + 48 * i, &k, &g, &st, m2, cn, &op, col,
                    &dep, rc, NULL, NULL, NULL);
        if (st.culled) continue;
        for (int q = 0; q < 9; q++) {
            double bq = b2d[9 * i + q];
            if (!(bq > 0)) continue;
            double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            double pz[6] = {0, 0, 0, 0, 0, 0};
            e[q] = bq;
            project_bwd_item(&st, e, sh + 48 * i, &k, &g, gm, &gl, gls, gq, gsh, pz);
            for (int c = 0; c < 3; c++) b_mean[3 * i + c] += fabs(gm[c]), b_logscale[3 * i + c] += fabs(gls[c]);
            for (int c = 0; c < 4; c++) b_quat[4 * i + c] += fabs(gq[c]);
            for (int c = 0; c < 48; c++) b_sh[48 * i + c] += fabs(gsh[c]);
            b_logit[i] += fabs(gl);
            for (int c = 0; c < 6; c++) item_pose[12 * i + c] += fabs(pz[c]);
        }
        if (g2d) {
            double pz[6] = {0, 0, 0, 0, 0, 0};
            project_bwd_item(&st, g2d + 9 * i, sh + 48 * i, &k, &g, gm, &gl, gls, gq, gsh, pz);
            for (int c = 0; c < 6; c++) item_pose[12 * i + 6 + c] = fabs(pz[c]);
        }
    }
    for (int c = 0; c < 6; c++) b_pose[c] = 0, pose_absum[c] = 0;
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < 6; c++) b_pose[c] += item_pose[12 * i + c], pose_absum[c] += item_pose[12 * i + 6 + c];
    free(item_pose);
}

/* Per-item Jacobian of the view's pose gradient with respect to the item's 2D
 * adjoint: jac[54 i + 9 c + q] = d pose_c / d g2d_q (zeros for culled items).
 * The projection adjoint is linear in g2d, so column q is the item adjoint of
 * the unit vector e_q. */
void or_pose_jacobian(int64_t n, const double* mean_opa, const double* scale, const double* quat,
                      const double* sh, const double* cam, const double* cfg, double* jac) {
    Cam k = read_cam(cam);
    Cfg g = read_cfg(cfg);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        ProjState st;
        double m2[2], cn[3], op, col[3], dep;
        int32_t rc[4];
        double gm[3], gl, gls[3], gq[4], gsh[48];
        for (int c = 0; c < 54; c++) jac[54 * i + c] = 0;
        project_one(0, mean_opa + 4 * i, scale + 4 * i, quat + 4 * i, sh + 48 * i, &k, &g, &st, m2, cn, &op, col,
                    &dep, rc, NULL, NULL, NULL);
        if (st.culled) continue;
        for (int q = 0; q < 9; q++) {
            double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            double pz[6] = {0, 0, 0, 0, 0, 0};
            e[q] = 1.0;
            project_bwd_item(&st, e, sh + 48 * i, &k, &g, gm, &gl, gls, gq, gsh, pz);
            for (int c = 0; c < 6; c++) jac[54 * i + 9 * c + q] = pz[c];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Tolerance bounds for an FP32 implementation of the compositing adjoint.
 *
 * Two effects move an FP32 result away from or_render_bwd's FP64 value by
 * more than a relative tolerance can express, and both are computed here from
 * the oracle's own state (nothing from the implementation under test):
 *
 * (1) Decisions within their margin (alpha_min, the 0.99 clamp, the exponent
 *     sign, termination, depth near-ties, and tile-list membership where a
 *     rect edge lies within the margin of a tile boundary) may go either way.
 *     Each pixel's decision is forced to its other branch on its own (depth
 *     near-ties: the two Gaussians swapped), the pixel's adjoint is
 *     recomputed, and |change| is accumulated per item and component
 *     (b_flip). A list membership concerns a whole tile, so its change is
 *     summed over the tile's pixels before the absolute value. With the
 *     per-item pose Jacobian (or_pose_jacobian), pose_flip[6] accumulates
 *     |sum over items of J (change)| per flip: the most the view's pose
 *     gradient can move when any subset of the flagged decisions flips.
 * (2) FP32 rounding of a back-to-front adjoint: the transmittance in front of
 *     a Gaussian is recovered from the stored final transmittance through the
 *     Gaussians behind it, so its relative error grows with each of them by
 *     alpha/(1-alpha) times the alpha uncertainty plus two roundings, on top
 *     of the forward's own accumulated error. The first-order error bound e of
 *     each contribution follows from that, from the exponent's uncertainty and
 *     from the splat centre's last bits. Summed as |e| these bounds grow with
 *     the number of pixels while the errors themselves, of varying sign,
 *     largely cancel; b_fp32 is therefore the root of the sum of e^2 per item
 *     and component (the scale of a sum of independent errors, as in
 *     probabilistic rounding-error analysis), and pose_fp32 the same for the
 *     pose through |J|. Callers multiply it by the confidence factor they
 *     choose.
 * amb_in [H*W] (may be NULL) marks pixels whose decisions are not modelled:
 * there |contribution| itself counts in b_flip.
 * memb [n_memb][3] = (tile, item, group) triples whose membership is
 * uncertain, sorted by tile; items absent from the tile's list are inserted in
 * (depth key, id) order. The memberships of one group change together (the
 * tiles of one rect edge, or of a Gaussian that may vanish or appear), so
 * their pose changes are summed with sign before the absolute value. Outputs
 * are overwritten.
 * ------------------------------------------------------------------------- */
#define MAX_FLAGS 64
typedef struct {
    int64_t cap;
    Contrib* rec;
    Contrib* recf;
    double *cb, *c0, *cf, *acc;
    int32_t* lst;
} BScratch;

static void bs_reserve(BScratch* s, int64_t len) {
    if (len + 2 <= s->cap) return;
    s->cap = len + 2;
    s->rec = (Contrib*)realloc(s->rec, sizeof(Contrib) * s->cap);
    s->recf = (Contrib*)realloc(s->recf, sizeof(Contrib) * s->cap);
    s->cb = (double*)realloc(s->cb, sizeof(double) * 9 * s->cap);
    s->c0 = (double*)realloc(s->c0, sizeof(double) * 9 * s->cap);
    s->cf = (double*)realloc(s->cf, sizeof(double) * 9 * s->cap);
    s->acc = (double*)realloc(s->acc, sizeof(double) * 9 * s->cap);
    s->lst = (int32_t*)realloc(s->lst, sizeof(int32_t) * s->cap);
}

/* contributions of the pixel under list lst (length len) and optional flip,
 * scattered by position into out[9 * (len + 1)] after map (position in lst ->
 * position in the caller's numbering; NULL = identity). Returns the last
 * position touched + 1 in the caller's numbering. */
static int64_t pixel_by_position(const Cfg* g, double px, double py, const int32_t* lst, int64_t len,
                                 const double* mean2d, const double* conic, const double* opac, const double* rgb,
                                 const double* depth, const double* gC, const Flag* flip, const int64_t* map,
                                 int64_t out_len, Contrib* rec, double* cb, double* out) {
    double col[3], Tf;
    int32_t nc;
    uint8_t a = 0;
    int nr = composite_pixel(g, px, py, lst, len, mean2d, conic, opac, rgb, depth, col, &Tf, &nc, &a, rec, NULL,
                             flip, NULL, 0, NULL);
    pixel_contribs(g, px, py, rec, nr, Tf, mean2d, conic, rgb, gC, cb);
    for (int64_t q = 0; q < 9 * out_len; q++) out[q] = 0;
    int64_t hi = 0;
    for (int r = 0; r < nr; r++) {
        int64_t j = map ? map[rec[r].j] : rec[r].j;
        for (int q = 0; q < 9; q++) out[9 * j + q] = cb[9 * r + q];
        if (j + 1 > hi) hi = j + 1;
    }
    return hi;
}

static void pose_of(const double* jac, int32_t id, const double* v, double* d) {
    for (int c = 0; c < 6; c++) {
        double s = 0;
        for (int q = 0; q < 9; q++) s += jac[54 * (int64_t)id + 9 * c + q] * v[q];
        d[c] += s;
    }
}

void or_render_bwd_bounds(const double* cam, const double* cfg, const int64_t* tile_start, const int32_t* ids,
                          const double* mean2d, const double* conic, const double* opac, const double* rgb,
                          const double* depth, const float* depth_key, const double* dL_dcolor, int64_t n,
                          const int64_t* memb, int64_t n_memb, const uint8_t* amb_in, const double* jac,
                          double* b_flip, double* b_fp32, double* pose_flip, double* pose_fp32) {
    Cam k = read_cam(cam);
    Cfg g = read_cfg(cfg);
    int T = g.tile, tx = (k.W + T - 1) / T, ty = (k.H + T - 1) / T;
    int64_t HW = (int64_t)k.W * k.H, nt = (int64_t)tx * ty;
    int64_t P = tile_start[nt];
    const double u = ldexp(1.0, -24);
    double* pf = (double*)calloc((size_t)(P > 0 ? P : 1) * 9, sizeof(double));
    double* p32 = (double*)calloc((size_t)(P > 0 ? P : 1) * 9, sizeof(double));
    double* pm = (double*)calloc((size_t)(n_memb > 0 ? n_memb : 1) * 9, sizeof(double));
    double* tpose = (double*)calloc((size_t)(nt > 0 ? nt : 1) * 12, sizeof(double));
    int64_t* mstart = (int64_t*)calloc((size_t)nt + 1, sizeof(int64_t));
    double* mpose = (double*)calloc((size_t)(n_memb > 0 ? n_memb : 1) * 6, sizeof(double));
    int64_t n_group = 0;
    for (int64_t m = 0; m < n_memb; m++) {
        mstart[memb[3 * m] + 1]++;
        if (memb[3 * m + 2] + 1 > n_group) n_group = memb[3 * m + 2] + 1;
    }
    for (int64_t t = 0; t < nt; t++) mstart[t + 1] += mstart[t];
#pragma omp parallel
    {
        BScratch s = {0, NULL, NULL, NULL, NULL, NULL, NULL, NULL};
        int64_t* map = NULL;
        int64_t map_cap = 0;
        Flag flags[MAX_FLAGS];
#pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < nt; t++) {
            int64_t b0 = tile_start[t], len = tile_start[t + 1] - b0;
            const int32_t* L = ids + b0;
            bs_reserve(&s, len);
            if (len + 2 > map_cap) { map_cap = len + 2; map = (int64_t*)realloc(map, sizeof(int64_t) * map_cap); }
            double* tp = tpose + 12 * t;
            int x0 = (int)(t % tx) * T, y0 = (int)(t / tx) * T;
            /* per-pixel decisions and FP32 rounding */
            for (int y = y0; y < y0 + T && y < k.H; y++)
                for (int x = x0; x < x0 + T && x < k.W; x++) {
                    int64_t pix = (int64_t)y * k.W + x;
                    double px = x + 0.5, py = y + 0.5, col[3], Tf;
                    double gC[3] = {dL_dcolor[pix], dL_dcolor[HW + pix], dL_dcolor[2 * HW + pix]};
                    int32_t nc;
                    uint8_t a = 0;
                    int nfl = 0;
                    int nr = composite_pixel(&g, px, py, L, len, mean2d, conic, opac, rgb, depth, col, &Tf, &nc, &a,
                                             s.rec, NULL, NULL, flags, MAX_FLAGS, &nfl);
                    pixel_contribs(&g, px, py, s.rec, nr, Tf, mean2d, conic, rgb, gC, s.cb);
                    /* (2) FP32 rounding */
                    double U = 0, dmax = 0;
                    for (int r = 0; r < nr; r++) {
                        U += s.rec[r].alpha / (1.0 - s.rec[r].alpha) * s.rec[r].dpow + 2 * u;
                        if (s.rec[r].dpow > dmax) dmax = s.rec[r].dpow;
                    }
                    double total[3] = {0, 0, 0};
                    for (int r = 0; r < nr; r++)
                        for (int ch = 0; ch < 3; ch++) total[ch] += s.rec[r].alpha * s.rec[r].T * rgb[3 * s.rec[r].id + ch];
                    double prefix[3] = {0, 0, 0};
                    double back = 0;
                    for (int r = nr - 1; r >= 0; r--) back += s.rec[r].alpha / (1.0 - s.rec[r].alpha) * s.rec[r].dpow + 4 * u;
                    for (int r = 0; r < nr; r++) {
                        const Contrib* c = &s.rec[r];
                        int32_t id = c->id;
                        /* relative error of the recovered T_r: forward error of T_final plus the
                         * recovery through every Gaussian from r to the back */
                        double al = c->alpha, tr = c->T;
                        double rel = U + back + (1.0 + al / (1.0 - al)) * c->dpow + ldexp(1.0, -20) + 64 * u + (nr - r) * u;
                        double mag = 0;
                        for (int ch = 0; ch < 3; ch++) {
                            double ci = rgb[3 * id + ch];
                            prefix[ch] += al * tr * ci;
                            double after = total[ch] - prefix[ch];
                            mag += fabs(gC[ch]) * (tr * fabs(ci) + (fabs(after) + fabs(Tf * g.bg[ch])) / (1.0 - al));
                        }
                        double e_da = mag * rel + dmax * mag;
                        const double* o = s.cb + 9 * r;
                        double b[9];
                        for (int ch = 0; ch < 3; ch++) b[6 + ch] = fabs(o[6 + ch]) * (rel + 4 * u);
                        for (int q = 0; q < 6; q++) b[q] = 0;
                        if (!c->clamped) {
                            double dx = px - mean2d[2 * id], dy = py - mean2d[2 * id + 1];
                            double ca = conic[3 * id], cbb = conic[3 * id + 1], cc = conic[3 * id + 2];
                            double ulp = 4.0 * ldexp(fmax(1.0, fmax(fabs(mean2d[2 * id]), fabs(mean2d[2 * id + 1]))), -24);
                            double f[5] = {ca * dx + cbb * dy, cbb * dx + cc * dy, -0.5 * dx * dx, -dx * dy, -0.5 * dy * dy};
                            double fe[5] = {(fabs(ca) + fabs(cbb)) * ulp + 1e-5 * (fabs(ca * dx) + fabs(cbb * dy)),
                                            (fabs(cbb) + fabs(cc)) * ulp + 1e-5 * (fabs(cbb * dx) + fabs(cc * dy)),
                                            fabs(dx) * ulp, (fabs(dx) + fabs(dy)) * ulp, fabs(dy) * ulp};
                            /* |dalpha| from the opacity share: o[5] = dalpha g */
                            double dalpha = c->g > 0 ? fabs(o[5]) / c->g : 0;
                            double e_dp = e_da * c->og + dalpha * c->og * c->dpow;
                            double dpw = dalpha * c->og;
                            for (int q = 0; q < 5; q++) b[q] = e_dp * fabs(f[q]) + dpw * fe[q] + 4 * u * fabs(o[q]);
                            b[5] = e_da * c->g + dalpha * c->g * c->dpow + 4 * u * fabs(o[5]);
                        }
                        for (int q = 0; q < 9; q++) p32[9 * (b0 + c->j) + q] += b[q] * b[q];
                        if (jac) {
                            for (int cc6 = 0; cc6 < 6; cc6++) {
                                double sacc = 0;
                                for (int q = 0; q < 9; q++) sacc += fabs(jac[54 * (int64_t)id + 9 * cc6 + q]) * b[q];
                                tp[6 + cc6] += sacc * sacc;
                            }
                        }
                        back -= c->alpha / (1.0 - c->alpha) * c->dpow + 4 * u;
                    }
                    /* scatter the pixel's contributions by list position */
                    for (int64_t q = 0; q < 9 * (len + 1); q++) s.c0[q] = 0;
                    int64_t hi0 = 0;
                    for (int r = 0; r < nr; r++) {
                        for (int q = 0; q < 9; q++) s.c0[9 * s.rec[r].j + q] = s.cb[9 * r + q];
                        hi0 = s.rec[r].j + 1;
                    }
                    if (amb_in && amb_in[pix]) {
                        double d[6] = {0, 0, 0, 0, 0, 0};
                        for (int r = 0; r < nr; r++) {
                            int64_t j = s.rec[r].j;
                            for (int q = 0; q < 9; q++) pf[9 * (b0 + j) + q] += fabs(s.c0[9 * j + q]);
                            if (jac)
                                for (int cc6 = 0; cc6 < 6; cc6++)
                                    for (int q = 0; q < 9; q++)
                                        d[cc6] += fabs(jac[54 * (int64_t)L[j] + 9 * cc6 + q] * s.c0[9 * j + q]);
                        }
                        for (int cc6 = 0; cc6 < 6; cc6++) tp[cc6] += d[cc6];
                    }
                    /* (1) every recorded decision flipped on its own */
                    for (int f = 0; f < nfl; f++) {
                        int64_t hi;
                        if (flags[f].kind == FL_DEPTH) {
                            int64_t j1 = flags[f].j, j2 = flags[f].j2;
                            memcpy(s.lst, L, sizeof(int32_t) * (size_t)len);
                            s.lst[j1] = L[j2];
                            s.lst[j2] = L[j1];
                            for (int64_t j = 0; j < len; j++) map[j] = j;
                            map[j1] = j2;
                            map[j2] = j1;
                            hi = pixel_by_position(&g, px, py, s.lst, len, mean2d, conic, opac, rgb, depth, gC, NULL,
                                                   map, len + 1, s.recf, s.cb, s.cf);
                        } else {
                            hi = pixel_by_position(&g, px, py, L, len, mean2d, conic, opac, rgb, depth, gC, &flags[f],
                                                   NULL, len + 1, s.recf, s.cb, s.cf);
                        }
                        if (hi0 > hi) hi = hi0;
                        double d[6] = {0, 0, 0, 0, 0, 0};
                        for (int64_t j = 0; j < hi; j++) {
                            double dv[9];
                            int nz = 0;
                            for (int q = 0; q < 9; q++) {
                                dv[q] = s.cf[9 * j + q] - s.c0[9 * j + q];
                                nz |= dv[q] != 0;
                            }
                            if (!nz) continue;
                            for (int q = 0; q < 9; q++) pf[9 * (b0 + j) + q] += fabs(dv[q]);
                            if (jac) pose_of(jac, L[j], dv, d);
                        }
                        for (int cc6 = 0; cc6 < 6; cc6++) tp[cc6] += fabs(d[cc6]);
                    }
                }
            /* (1) uncertain list memberships of this tile, one at a time over the whole tile */
            for (int64_t m = mstart[t]; m < mstart[t + 1]; m++) {
                int32_t item = (int32_t)memb[3 * m + 1];
                int64_t jr = -1;
                for (int64_t j = 0; j < len; j++)
                    if (L[j] == item) { jr = j; break; }
                int64_t len2;
                if (jr >= 0) { /* remove it */
                    len2 = len - 1;
                    for (int64_t j = 0, w = 0; j < len; j++)
                        if (j != jr) { s.lst[w] = L[j]; map[w] = j; w++; }
                } else { /* insert it in (depth key, id) order */
                    uint32_t kb;
                    memcpy(&kb, &depth_key[item], 4);
                    int64_t ji = 0;
                    while (ji < len) {
                        uint32_t kj;
                        memcpy(&kj, &depth_key[L[ji]], 4);
                        if (kj > kb || (kj == kb && L[ji] > item)) break;
                        ji++;
                    }
                    len2 = len + 1;
                    for (int64_t j = 0, w = 0; w < len2; w++) {
                        if (w == ji) { s.lst[w] = item; map[w] = len; }
                        else { s.lst[w] = L[j]; map[w] = j; j++; }
                    }
                }
                for (int64_t q = 0; q < 9 * (len + 1); q++) s.acc[q] = 0;
                for (int y = y0; y < y0 + T && y < k.H; y++)
                    for (int x = x0; x < x0 + T && x < k.W; x++) {
                        int64_t pix = (int64_t)y * k.W + x;
                        double px = x + 0.5, py = y + 0.5;
                        double gC[3] = {dL_dcolor[pix], dL_dcolor[HW + pix], dL_dcolor[2 * HW + pix]};
                        pixel_by_position(&g, px, py, L, len, mean2d, conic, opac, rgb, depth, gC, NULL, NULL, len + 1,
                                          s.rec, s.cb, s.c0);
                        pixel_by_position(&g, px, py, s.lst, len2, mean2d, conic, opac, rgb, depth, gC, NULL, map,
                                          len + 1, s.recf, s.cb, s.cf);
                        for (int64_t q = 0; q < 9 * (len + 1); q++) s.acc[q] += s.cf[q] - s.c0[q];
                    }
                double d[6] = {0, 0, 0, 0, 0, 0};
                for (int64_t j = 0; j < len; j++) {
                    for (int q = 0; q < 9; q++) pf[9 * (b0 + j) + q] += fabs(s.acc[9 * j + q]);
                    if (jac) pose_of(jac, L[j], s.acc + 9 * j, d);
                }
                for (int q = 0; q < 9; q++) pm[9 * m + q] = fabs(s.acc[9 * len + q]);
                if (jac && jr < 0) pose_of(jac, item, s.acc + 9 * len, d);
                for (int cc6 = 0; cc6 < 6; cc6++) mpose[6 * m + cc6] = d[cc6];
            }
        }
        free(s.rec); free(s.recf); free(s.cb); free(s.c0); free(s.cf); free(s.acc); free(s.lst); free(map);
    }
    for (int64_t i = 0; i < 9 * n; i++) b_flip[i] = 0, b_fp32[i] = 0;
    for (int64_t j = 0; j < P; j++)
        for (int q = 0; q < 9; q++) {
            b_flip[9 * (int64_t)ids[j] + q] += pf[9 * j + q];
            b_fp32[9 * (int64_t)ids[j] + q] += p32[9 * j + q];
        }
    for (int64_t i = 0; i < 9 * n; i++) b_fp32[i] = sqrt(b_fp32[i]);
    for (int64_t m = 0; m < n_memb; m++)
        for (int q = 0; q < 9; q++) b_flip[9 * memb[3 * m + 1] + q] += pm[9 * m + q];
    for (int c = 0; c < 6; c++) pose_flip[c] = 0, pose_fp32[c] = 0;
    for (int64_t t = 0; t < nt; t++)
        for (int c = 0; c < 6; c++) pose_flip[c] += tpose[12 * t + c], pose_fp32[c] += tpose[12 * t + 6 + c];
    for (int c = 0; c < 6; c++) pose_fp32[c] = sqrt(pose_fp32[c]);
    double* gpose = (double*)calloc((size_t)(n_group > 0 ? n_group : 1) * 6, sizeof(double));
    for (int64_t m = 0; m < n_memb; m++)
        for (int c = 0; c < 6; c++) gpose[6 * memb[3 * m + 2] + c] += mpose[6 * m + c];
    for (int64_t q = 0; q < n_group; q++)
        for (int c = 0; c < 6; c++) pose_flip[c] += fabs(gpose[6 * q + c]);
    free(gpose);
    free(mpose);
    free(pf); free(p32); free(pm); free(tpose); free(mstart);
}

/* ---------------------------------------------------------------------------
 * Direct spawn sampling (Sec. 4.2).
 *
 * P_L = min(|| LoG_sigma * I ||, 1)      (Eq. 1, norm over the RGB responses)
 * P~  = min(|| LoG_sigma * I~ ||, 1)     (Eq. 2, I~ the render from the new pose)
 * P_s = max(P_L - P~, 0)                 (Eq. 3)
 * The LoG kernel is the continuous Laplacian of the Gaussian n_sigma sampled at
 * integer offsets up to radius ceil(3 sigma), shifted to zero sum (so constant
 * regions respond 0); borders replicate. Computed here as a direct 2-D
 * convolution. The mask draws u = Philox4x32-10(counter = (pixel, frame, 0, 0),
 * key = seed) -> top 24 bits of word 0 / 2^24 and spawns iff u < P_s.
 * ------------------------------------------------------------------------- */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64
 * multiplications by M0, M1 with the key bumped by the Weyl constants W0, W1. */
void or_philox4x32_10(const uint32_t* ctr_in, const uint32_t* key_in, uint32_t* out) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double log_kernel_value(double x, double y, double s) {
    double r2 = x * x + y * y, s2 = s * s;
    return (r2 - 2 * s2) / (s2 * s2) * exp(-r2 / (2 * s2)) / (2 * PI_D * s2);
}

/* Fills the (2R+1)^2 zero-sum sampled LoG kernel; returns R. */
int or_log_kernel(double sigma, double* k /* (2R+1)^2, R <= 12 */) {
    int R = (int)ceil(3 * sigma);
    int n = 2 * R + 1;
    double sum = 0;
    for (int j = -R; j <= R; j++)
        for (int i = -R; i <= R; i++) sum += (k[(j + R) * n + (i + R)] = log_kernel_value(i, j, sigma));
    for (int t = 0; t < n * n; t++) k[t] -= sum / (n * n);
    return R;
}

static void log_norm_map(const double* img, int W, int H, const double* k, int R, double* out) {
    int n = 2 * R + 1;
    int64_t HW = (int64_t)W * H;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < HW; p++) {
        int x = (int)(p % W), y = (int)(p / W);
        double acc2 = 0;
        for (int ch = 0; ch < 3; ch++) {
            double a = 0;
            for (int j = -R; j <= R; j++) {
                int yy = y + j < 0 ? 0 : (y + j >= H ? H - 1 : y + j);
                for (int i = -R; i <= R; i++) {
                    int xx = x + i < 0 ? 0 : (x + i >= W ? W - 1 : x + i);
                    a += k[(j + R) * n + (i + R)] * img[ch * HW + (int64_t)yy * W + xx];
                }
            }
            acc2 += a * a;
        }
        double v = sqrt(acc2);
        out[p] = v < 1 ? v : 1;
    }
}

/* image, render: [3][H][W] in [0, 1] (render may be NULL: nothing rendered yet,
 * P~ = 0). Outputs per pixel: p_l, p_pen, p_s, u (the uniform draw), mask, and
 * amb = 1 where |u - P_s| is within margin (the FP32 path may decide either way). */
void or_spawn_maps(const double* image, const double* render, int W, int H, double sigma, uint64_t seed,
                   uint32_t frame, double margin, double* p_l, double* p_pen, double* p_s, double* u, uint8_t* mask,
                   uint8_t* amb) {
    double k[25 * 25];
    int R = or_log_kernel(sigma, k);
    int64_t HW = (int64_t)W * H;
    log_norm_map(image, W, H, k, R, p_l);
    if (render) log_norm_map(render, W, H, k, R, p_pen);
    else for (int64_t p = 0; p < HW; p++) p_pen[p] = 0;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < HW; p++) {
        double d = p_l[p] - p_pen[p];
        p_s[p] = d > 0 ? d : 0;
        uint32_t ctr[4] = {(uint32_t)p, frame, 0u, 0u}, o[4];
        or_philox4x32_10(ctr, key, o);
        u[p] = (double)(o[0] >> 8) / 16777216.0;
        mask[p] = u[p] < p_s[p];
        amb[p] = fabs(u[p] - p_s[p]) < margin;
    }
}

/* u[p] = (word 0 of Philox4x32-10(counter (p, c1, c2, 0), key seed)) >> 8, / 2^24,
 * for p = 0 .. n-1: the uniform draws of the spawn masks. */
void or_philox_uniforms(int64_t n, uint32_t c1, uint32_t c2, uint64_t seed, double* u) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) {
        uint32_t ctr[4] = {(uint32_t)p, c1, c2, 0u}, o[4];
        or_philox4x32_10(ctr, key, o);
        u[p] = (double)(o[0] >> 8) / 16777216.0;
    }
}
