/*
 * tsplat_oracle.c -- plain, slow CPU oracle for the latent-Gaussian
 * splatting path of Tele-Aloha (Sec. 4.2, "Neural Rasterization via 3DGS").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header or constant table with the CUDA library.
 *
 * What the method computes, and what this file restates step by step:
 *   Sec. 4.2, latent Gaussian record: each point has a position x_i, a
 *     latent feature f_i (d channels), a scale s_i and an opacity alpha_i;
 *     the paper sets the rotation to the identity.  Rotations are taken here
 *     as an input (identity reproduces the paper).
 *   Sec. 4.2, lifting: foreground pixels of each source depth map are
 *     unprojected with the source camera Pi to pixel-aligned Gaussians.
 *   Sec. 4.2, render equation F_novel = R_G({G}, Pi_novel): the
 *     differentiable Gaussian splatting rasterizer of Kerbl et al. 2023 that
 *     the paper cites: EWA projection of each Gaussian to a 2D conic,
 *     binning to 16x16 tiles, ordering by (tile, depth), and front-to-back
 *     alpha compositing -- here of the latent features instead of colour.
 *
 * Precision.  Every function is IEEE double except the "key mode" (suffix
 * _f32), which evaluates the quantities that decide integers -- lifted
 * Gaussians, visibility, radius, tile rectangle, depth sort key -- in strict
 * single precision, one correctly rounded operation at a time, in the order
 * written.  The file must be compiled with -ffp-contract=off and without
 * -ffast-math so that no multiply-add is fused.
 *
 * Array layouts (all row-major, C order):
 *   camera  float[20]: fx fy cx cy width height R[9] t[3] z_near z_far,
 *           R,t world->camera (p_cam = R x + t); pixel (u,v) = (col,row)
 *           is centred at image coordinate (u,v).
 *   params  float[5] : lowpass alpha_max alpha_min t_min frustum_clamp.
 *   cov     6 values : s00 s01 s02 s11 s12 s22 of the symmetric 3x3.
 *   conic   3 values : (a, b, c) of the inverse 2x2 covariance [[a,b],[b,c]].
 *   rect    4 int32  : x0 y0 x1 y1 tile bounds, half open.
 *   F       C x H x W, A / T_final / last: H x W.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TILE 16

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * BF16 storage rounding: round-to-nearest-even of a float's upper 16 bits
 * (the storage format of the precision workload).  Finite inputs only.
 * ---------------------------------------------------------------------- */
void orc_round_bf16(int64_t n, const float *in, float *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &in[i], 4);
        uint32_t lsb = (u >> 16) & 1u;
        u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;
        memcpy(&out[i], &u, 4);
    }
}

/* ------------------------------------------------------------------------
 * Lifting (Sec. 4.2: positions unprojected from depth with Pi; foreground
 * pixels become pixel-aligned Gaussians).
 *
 * For pixel (u,v) with depth z of a camera with intrinsics (fx,fy,cx,cy)
 * and world->camera (R,t):
 *     x_cam   = z * ((u-cx)/fx, (v-cy)/fy, 1)
 *     x_world = R^T (x_cam - t)
 * The Gaussian's rotation R_g = R^T R(q) maps its local axes (given in the
 * source camera frame by the unit quaternion q = (w,x,y,z)) to the world,
 * and Sigma3D = R_g diag(s)^2 R_g^T.  Gaussians are numbered in
 * (row, column) order of the foreground pixels.
 * ---------------------------------------------------------------------- */
int64_t orc_lift_f64(int H, int W, int C, const float *depth, const uint8_t *mask,
                     const float *scale, const float *quat, const float *opac,
                     const float *feat, const float *cam,
                     double *mean, double *cov, double *op, double *ft)
{
    const double fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    double R[9], t[3];
    for (int k = 0; k < 9; ++k) R[k] = cam[6 + k];
    for (int k = 0; k < 3; ++k) t[k] = cam[15 + k];
    int64_t n = 0;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            int64_t p = (int64_t)v * W + u;
            if (mask && !mask[p]) continue;
            double z = depth[p];
            double xc[3] = {z * ((u - cx) / fx), z * ((v - cy) / fy), z};
            double d[3] = {xc[0] - t[0], xc[1] - t[1], xc[2] - t[2]};
            for (int i = 0; i < 3; ++i)  /* R^T d */
                mean[3 * n + i] = R[0 * 3 + i] * d[0] + R[1 * 3 + i] * d[1] + R[2 * 3 + i] * d[2];

            double w = 1, x = 0, y = 0, zq = 0;
            if (quat) { w = quat[4 * p]; x = quat[4 * p + 1]; y = quat[4 * p + 2]; zq = quat[4 * p + 3]; }
            double nq = sqrt(w * w + x * x + y * y + zq * zq);
            w /= nq; x /= nq; y /= nq; zq /= nq;
            double Rq[3][3] = {
                {1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y)},
                {2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x)},
                {2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)}};
            double M[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double rg = R[0 * 3 + i] * Rq[0][j] + R[1 * 3 + i] * Rq[1][j] + R[2 * 3 + i] * Rq[2][j];
                    M[i][j] = rg * (double)scale[3 * p + j];
                }
            static const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
            for (int e = 0; e < 6; ++e)
                cov[6 * n + e] = M[ii[e]][0] * M[jj[e]][0] + M[ii[e]][1] * M[jj[e]][1] + M[ii[e]][2] * M[jj[e]][2];
            op[n] = opac[p];
            for (int c = 0; c < C; ++c) ft[n * C + c] = feat[p * C + c];
            ++n;
        }
    return n;
}

/* Key-mode lifting: the same steps in strict single precision, one rounded
 * operation at a time, in exactly the order written. */
int64_t orc_lift_f32(int H, int W, int C, const float *depth, const uint8_t *mask,
                     const float *scale, const float *quat, const float *opac,
                     const float *feat, const float *cam,
                     float *mean, float *cov, float *op, float *ft)
{
    const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    const float *R = cam + 6, *t = cam + 15;
    int64_t n = 0;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            int64_t p = (int64_t)v * W + u;
            if (mask && !mask[p]) continue;
            float z = depth[p];
            float rx = ((float)u - cx) / fx;
            float ry = ((float)v - cy) / fy;
            float d0 = rx * z - t[0];
            float d1 = ry * z - t[1];
            float d2 = z - t[2];
            for (int i = 0; i < 3; ++i) {
                float s01 = R[0 * 3 + i] * d0 + R[1 * 3 + i] * d1;
                mean[3 * n + i] = s01 + R[2 * 3 + i] * d2;
            }
            float w = 1.0f, x = 0.0f, y = 0.0f, zq = 0.0f;
            if (quat) { w = quat[4 * p]; x = quat[4 * p + 1]; y = quat[4 * p + 2]; zq = quat[4 * p + 3]; }
            float nn = ((w * w + x * x) + y * y) + zq * zq;
            float nq = sqrtf(nn);
            w = w / nq; x = x / nq; y = y / nq; zq = zq / nq;
            float Rq[3][3];
            Rq[0][0] = 1.0f - 2.0f * (y * y + zq * zq);
            Rq[0][1] = 2.0f * (x * y - w * zq);
            Rq[0][2] = 2.0f * (x * zq + w * y);
            Rq[1][0] = 2.0f * (x * y + w * zq);
            Rq[1][1] = 1.0f - 2.0f * (x * x + zq * zq);
            Rq[1][2] = 2.0f * (y * zq - w * x);
            Rq[2][0] = 2.0f * (x * zq - w * y);
            Rq[2][1] = 2.0f * (y * zq + w * x);
            Rq[2][2] = 1.0f - 2.0f * (x * x + y * y);
            float M[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    float rg = (R[0 * 3 + i] * Rq[0][j] + R[1 * 3 + i] * Rq[1][j]) + R[2 * 3 + i] * Rq[2][j];
                    M[i][j] = rg * scale[3 * p + j];
                }
            static const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
            for (int e = 0; e < 6; ++e)
                cov[6 * n + e] = (M[ii[e]][0] * M[jj[e]][0] + M[ii[e]][1] * M[jj[e]][1]) + M[ii[e]][2] * M[jj[e]][2];
            op[n] = opac[p];
            for (int c = 0; c < C; ++c) ft[n * C + c] = feat[p * C + c];
            ++n;
        }
    return n;
}

/* ------------------------------------------------------------------------
 * EWA projection (the cited 3DGS rasterizer's preprocessing step).
 *
 *   p = R x + t (target camera); visible iff z_near < p_z < z_far.
 *   Perspective Jacobian at p, with x/z and y/z clamped to
 *   +-frustum_clamp * tan(half field of view) (tan = 0.5 W / fx):
 *       J = [[fx/p_z, 0, -fx t_x/p_z^2], [0, fy/p_z, -fy t_y/p_z^2]]
 *   Sigma2D = (J R) Sigma3D (J R)^T + lowpass * I
 *   det = a c - b^2; a non-positive or non-finite det culls the Gaussian.
 *   conic = (c, -b, a) / det
 *   lambda_max = m + sqrt(max(0.1, m^2 - det)), m = (a + c)/2
 *   radius r = ceil(3 sqrt(lambda_max))
 *   mean2D mu = (fx p_x / p_z + cx, fy p_y / p_z + cy)
 *   tile rect = [floor((mu - r)/16), floor((mu + r + 15)/16)) clamped to
 *   the tile grid; an empty rect culls the Gaussian.
 *   The depth key is the bit pattern of p_z (an order-preserving code for
 *   positive floats); culled Gaussians get key 0xFFFFFFFF and no tiles.
 * ---------------------------------------------------------------------- */
void orc_project_f32(int64_t n, const float *mean, const float *cov, const float *cam,
                     const float *par, int32_t *rect, int32_t *ntiles, uint32_t *dkey,
                     float *radius, float *mu, float *conic)
{
    const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    const int W = (int)cam[4], H = (int)cam[5];
    const float *R = cam + 6, *t = cam + 15;
    const float znear = cam[18], zfar = cam[19];
    const float lp = par[0], clampf = par[4];
    const int tx_n = (W + TILE - 1) / TILE, ty_n = (H + TILE - 1) / TILE;
    const float limx = clampf * ((0.5f * (float)W) / fx);
    const float limy = clampf * ((0.5f * (float)H) / fy);

    for (int64_t i = 0; i < n; ++i) {
        const float x = mean[3 * i], y = mean[3 * i + 1], z = mean[3 * i + 2];
        float px = ((R[0] * x + R[1] * y) + R[2] * z) + t[0];
        float py = ((R[3] * x + R[4] * y) + R[5] * z) + t[1];
        float pz = ((R[6] * x + R[7] * y) + R[8] * z) + t[2];
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        ntiles[i] = 0; dkey[i] = 0xFFFFFFFFu; radius[i] = 0.0f;
        mu[2 * i] = mu[2 * i + 1] = 0.0f;
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0.0f;
        if (!(pz > znear && pz < zfar)) continue;

        float txz = fminf(limx, fmaxf(-limx, px / pz));
        float tyz = fminf(limy, fmaxf(-limy, py / pz));
        float tx = txz * pz, ty = tyz * pz;
        float pz2 = pz * pz;
        float j00 = fx / pz, j02 = -((fx * tx) / pz2);
        float j11 = fy / pz, j12 = -((fy * ty) / pz2);
        float T[2][3];
        for (int j = 0; j < 3; ++j) {
            T[0][j] = j00 * R[0 * 3 + j] + j02 * R[2 * 3 + j];
            T[1][j] = j11 * R[1 * 3 + j] + j12 * R[2 * 3 + j];
        }
        const float *cv = cov + 6 * i;
        float V[3][3] = {{cv[0], cv[1], cv[2]}, {cv[1], cv[3], cv[4]}, {cv[2], cv[4], cv[5]}};
        float U[2][3];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k)
                U[r][k] = (T[r][0] * V[0][k] + T[r][1] * V[1][k]) + T[r][2] * V[2][k];
        float s00 = (U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2];
        float s01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2];
        float s11 = (U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2];
        float a = s00 + lp, b = s01, c = s11 + lp;
        float det = a * c - b * b;
        if (!(det > 0.0f) || !isfinite(det)) continue;
        float mid = 0.5f * (a + c);
        float disc = fmaxf(0.1f, mid * mid - det);
        float lam = mid + sqrtf(disc);
        float r = ceilf(3.0f * sqrtf(lam));
        float mx = (fx * px) / pz + cx;
        float my = (fy * py) / pz + cy;
        float fx0 = floorf((mx - r) / 16.0f), fx1 = floorf(((mx + r) + 15.0f) / 16.0f);
        float fy0 = floorf((my - r) / 16.0f), fy1 = floorf(((my + r) + 15.0f) / 16.0f);
        int x0 = (int)fminf((float)tx_n, fmaxf(0.0f, fx0));
        int x1 = (int)fminf((float)tx_n, fmaxf(0.0f, fx1));
        int y0 = (int)fminf((float)ty_n, fmaxf(0.0f, fy0));
        int y1 = (int)fminf((float)ty_n, fmaxf(0.0f, fy1));
        int nt = (x1 - x0) * (y1 - y0);
        if (nt <= 0) continue;
        rect[4 * i] = x0; rect[4 * i + 1] = y0; rect[4 * i + 2] = x1; rect[4 * i + 3] = y1;
        ntiles[i] = nt;
        uint32_t kb;
        memcpy(&kb, &pz, 4);
        dkey[i] = kb;
        radius[i] = r;
        mu[2 * i] = mx; mu[2 * i + 1] = my;
        conic[3 * i] = c / det; conic[3 * i + 1] = -(b / det); conic[3 * i + 2] = a / det;
    }
}

/* Point z-buffer.  Tele-Aloha lifts one view's depth map to points and
 * rasterizes them into other cameras, reading the z-buffer out (Sec. 4.1,
 * cascaded disparity initialisation), and warps the predicted depth maps
 * onto the novel view (Sec. 4.3, fused depth).  A point is the Gaussian
 * mean: its camera-space depth pz and image position (mx, my) follow the
 * single-precision operations of orc_project_f32; it lands on the pixel whose
 * centre is nearest, (floor(mx + 0.5), floor(my + 0.5)), when pz lies in
 * (z_near, z_far) and the pixel is inside the image.  Each pixel keeps the
 * point of smallest pz (FP32 bits compared as integers, the same order for
 * positive depths), the lowest id among equal depths.
 *   depth: H*W f32, 0 where no point landed; id: H*W int32, -1 there. */
void orc_zbuffer(int64_t n, const float *mean, const float *cam, float *depth, int32_t *id)
{
    const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    const int W = (int)cam[4], H = (int)cam[5];
    const float *R = cam + 6, *t = cam + 15;
    const float znear = cam[18], zfar = cam[19];
    uint32_t *best = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)W * (size_t)H);
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
        depth[p] = 0.0f;
        id[p] = -1;
        best[p] = 0xFFFFFFFFu;
    }
    for (int64_t i = 0; i < n; ++i) {
        const float x = mean[3 * i], y = mean[3 * i + 1], z = mean[3 * i + 2];
        const float px = ((R[0] * x + R[1] * y) + R[2] * z) + t[0];
        const float py = ((R[3] * x + R[4] * y) + R[5] * z) + t[1];
        const float pz = ((R[6] * x + R[7] * y) + R[8] * z) + t[2];
        if (!(pz > znear && pz < zfar)) continue;
        const float mx = (fx * px) / pz + cx;
        const float my = (fy * py) / pz + cy;
        const float fu = floorf(mx + 0.5f), fv = floorf(my + 0.5f);
        if (!(fu >= 0.0f && fu < (float)W && fv >= 0.0f && fv < (float)H)) continue;
        const int64_t p = (int64_t)fv * W + (int64_t)fu;
        uint32_t bits;
        memcpy(&bits, &pz, 4);
        if (bits < best[p]) {  /* ids arrive in increasing order: ties keep the first */
            best[p] = bits;
            depth[p] = pz;
            id[p] = (int32_t)i;
        }
    }
    free(best);
}

/* The same projection in double precision (used for the compositing
 * values; binning decisions come from the key mode above).  `visible` is
 * set when the double-precision determinant is positive and finite. */
void orc_project_f64(int64_t n, const double *mean, const double *cov, const float *cam,
                     const float *par, double *mu, double *conic, double *depth, uint8_t *visible)
{
    const double fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    const double W = cam[4], H = cam[5];
    double R[9], t[3];
    for (int k = 0; k < 9; ++k) R[k] = cam[6 + k];
    for (int k = 0; k < 3; ++k) t[k] = cam[15 + k];
    const double lp = par[0], clampv = par[4];
    const double limx = clampv * (0.5 * W / fx), limy = clampv * (0.5 * H / fy);
    for (int64_t i = 0; i < n; ++i) {
        const double *m = mean + 3 * i;
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = R[3 * r] * m[0] + R[3 * r + 1] * m[1] + R[3 * r + 2] * m[2] + t[r];
        depth[i] = p[2];
        visible[i] = 0;
        mu[2 * i] = mu[2 * i + 1] = 0;
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
        if (!(p[2] > 0)) continue;
        double tx = fmin(limx, fmax(-limx, p[0] / p[2])) * p[2];
        double ty = fmin(limy, fmax(-limy, p[1] / p[2])) * p[2];
        double J[2][3] = {{fx / p[2], 0, -fx * tx / (p[2] * p[2])},
                          {0, fy / p[2], -fy * ty / (p[2] * p[2])}};
        double T[2][3];
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j < 3; ++j)
                T[r][j] = J[r][0] * R[0 * 3 + j] + J[r][1] * R[1 * 3 + j] + J[r][2] * R[2 * 3 + j];
        const double *cv = cov + 6 * i;
        double V[3][3] = {{cv[0], cv[1], cv[2]}, {cv[1], cv[3], cv[4]}, {cv[2], cv[4], cv[5]}};
        double S[2][2];
        for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += T[r][k] * V[k][l] * T[s][l];
                S[r][s] = acc;
            }
        double a = S[0][0] + lp, b = S[0][1], c = S[1][1] + lp;
        double det = a * c - b * b;
        mu[2 * i] = fx * p[0] / p[2] + cx;
        mu[2 * i + 1] = fy * p[1] / p[2] + cy;
        if (!(det > 0) || !isfinite(det)) continue;
        conic[3 * i] = c / det; conic[3 * i + 1] = -b / det; conic[3 * i + 2] = a / det;
        visible[i] = 1;
    }
}

/* Adjoint of orc_project_f64 (Sec. 4.2: the rasterizer is differentiated
 * end to end, so gradients reach the 3D Gaussians).  Given dL/dmu (N x 2)
 * and dL/d(conic) (N x 3, w.r.t. the stored (A, B, C) of
 * q = -(A dx^2 + 2 B dx dy + C dy^2) / 2), returns dL/dmean (N x 3, world
 * space) and dL/dcov (N x 6, w.r.t. the six stored entries of the
 * symmetric 3D covariance).  The chain: p = R x + t; mu = f p_xy / p_z + c;
 * J from p (x/z and y/z clamped: no gradient through a clamped ratio);
 * S = (J R) V (J R)^T + lowpass I; conic = S^-1.  Gaussians that the
 * forward culls (p_z <= 0, det <= 0) get zero. */
void orc_project_backward_f64(int64_t n, const double *mean, const double *cov, const float *cam,
                              const float *par, const double *g_mu, const double *g_conic,
                              double *g_mean, double *g_cov)
{
    const double fx = cam[0], fy = cam[1];
    const double W = cam[4], H = cam[5];
    double R[9], t[3];
    for (int k = 0; k < 9; ++k) R[k] = cam[6 + k];
    for (int k = 0; k < 3; ++k) t[k] = cam[15 + k];
    const double lp = par[0], clampv = par[4];
    const double limx = clampv * (0.5 * W / fx), limy = clampv * (0.5 * H / fy);
    for (int64_t i = 0; i < n; ++i) {
        double *gm = g_mean + 3 * i, *gc = g_cov + 6 * i;
        for (int k = 0; k < 3; ++k) gm[k] = 0;
        for (int k = 0; k < 6; ++k) gc[k] = 0;
        const double *m = mean + 3 * i;
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = R[3 * r] * m[0] + R[3 * r + 1] * m[1] + R[3 * r + 2] * m[2] + t[r];
        if (!(p[2] > 0)) continue;
        const double z = p[2];
        const double rx = p[0] / z, ry = p[1] / z;
        const int cx_in = rx > -limx && rx < limx, cy_in = ry > -limy && ry < limy;
        const double txz = fmin(limx, fmax(-limx, rx)), tyz = fmin(limy, fmax(-limy, ry));
        const double J00 = fx / z, J02 = -fx * txz / z, J11 = fy / z, J12 = -fy * tyz / z;
        double T[2][3];
        for (int j = 0; j < 3; ++j) {
            T[0][j] = J00 * R[0 * 3 + j] + J02 * R[2 * 3 + j];
            T[1][j] = J11 * R[1 * 3 + j] + J12 * R[2 * 3 + j];
        }
        const double *cv = cov + 6 * i;
        const double V[3][3] = {{cv[0], cv[1], cv[2]}, {cv[1], cv[3], cv[4]}, {cv[2], cv[4], cv[5]}};
        double VT0[3], VT1[3];  /* V t0, V t1 */
        for (int k = 0; k < 3; ++k) {
            VT0[k] = V[k][0] * T[0][0] + V[k][1] * T[0][1] + V[k][2] * T[0][2];
            VT1[k] = V[k][0] * T[1][0] + V[k][1] * T[1][1] + V[k][2] * T[1][2];
        }
        const double S00 = T[0][0] * VT0[0] + T[0][1] * VT0[1] + T[0][2] * VT0[2];
        const double S01 = T[0][0] * VT1[0] + T[0][1] * VT1[1] + T[0][2] * VT1[2];
        const double S11 = T[1][0] * VT1[0] + T[1][1] * VT1[1] + T[1][2] * VT1[2];
        const double a = S00 + lp, b = S01, c = S11 + lp;
        const double D = a * c - b * b;
        /* mean: mu = f p / z + c */
        double gp[3] = {fx / z * g_mu[2 * i], fy / z * g_mu[2 * i + 1],
                        -fx * p[0] / (z * z) * g_mu[2 * i] - fy * p[1] / (z * z) * g_mu[2 * i + 1]};
        if (D > 0 && isfinite(D)) {
            const double gA = g_conic[3 * i], gB = g_conic[3 * i + 1], gC = g_conic[3 * i + 2];
            const double D2 = D * D;
            /* A = c / D, B = -b / D, C = a / D, D = a c - b^2 */
            const double ga = -gA * c * c / D2 + gB * b * c / D2 + gC * (1.0 / D - a * c / D2);
            const double gb = gA * 2 * b * c / D2 + gB * (-1.0 / D - 2 * b * b / D2) + gC * 2 * a * b / D2;
            const double gcc = gA * (1.0 / D - a * c / D2) + gB * a * b / D2 - gC * a * a / D2;
            /* S00 = t0^T V t0, S01 = t0^T V t1, S11 = t1^T V t1 */
            static const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
            for (int e = 0; e < 6; ++e) {
                const int u = ii[e], v = jj[e];
                double d00 = T[0][u] * T[0][v], d01 = T[0][u] * T[1][v], d11 = T[1][u] * T[1][v];
                if (u != v) {
                    d00 += T[0][v] * T[0][u];
                    d01 += T[0][v] * T[1][u];
                    d11 += T[1][v] * T[1][u];
                }
                gc[e] = ga * d00 + gb * d01 + gcc * d11;
            }
            double gt0[3], gt1[3];
            for (int k = 0; k < 3; ++k) {
                gt0[k] = 2 * ga * VT0[k] + gb * VT1[k];
                gt1[k] = gb * VT0[k] + 2 * gcc * VT1[k];
            }
            double gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
            for (int k = 0; k < 3; ++k) {
                gJ00 += gt0[k] * R[0 * 3 + k];
                gJ02 += gt0[k] * R[2 * 3 + k];
                gJ11 += gt1[k] * R[1 * 3 + k];
                gJ12 += gt1[k] * R[2 * 3 + k];
            }
            /* J00 = fx / z; J02 = -fx txz / z with txz = p_x / z when not clamped */
            gp[2] += -fx / (z * z) * gJ00 - fy / (z * z) * gJ11;
            if (cx_in) {
                gp[0] += -fx / (z * z) * gJ02;
                gp[2] += 2 * fx * p[0] / (z * z * z) * gJ02;
            } else {
                gp[2] += fx * txz / (z * z) * gJ02;
            }
            if (cy_in) {
                gp[1] += -fy / (z * z) * gJ12;
                gp[2] += 2 * fy * p[1] / (z * z * z) * gJ12;
            } else {
                gp[2] += fy * tyz / (z * z) * gJ12;
            }
        }
        for (int k = 0; k < 3; ++k) gm[k] = R[0 * 3 + k] * gp[0] + R[1 * 3 + k] * gp[1] + R[2 * 3 + k] * gp[2];
    }
}

/* Adjoint of orc_lift_f64 for one view (Sec. 4.2: lifting with the source
 * camera; trained end to end, the gradients reach the encoder's depth,
 * scale, opacity and feature maps).  Gaussian n is the n-th foreground pixel
 * in row-major order.  Inputs dL/dmean (N x 3), dL/dcov (N x 6), dL/dopac
 * (N), dL/dfeat (N x C); outputs per pixel (zero outside the mask):
 * g_depth (H x W), g_scale (H x W x 3), g_quat (H x W x 4, w.r.t. the
 * unnormalised quaternion; may be NULL), g_opac (H x W), g_feat (H x W x C).
 * mean = Rs^T (z ray - ts), ray = ((u - cx)/fx, (v - cy)/fy, 1);
 * cov = M M^T with M = Rs^T R(q^) diag(s), q^ = q / |q|. */
void orc_lift_backward_f64(int H, int W, int C, const float *depth, const uint8_t *mask, const float *scale,
                           const float *quat, const float *cam, const double *g_mean, const double *g_cov,
                           const double *g_op, const double *g_ft, double *g_depth, double *g_scale,
                           double *g_quat, double *g_opac, double *g_feat)
{
    const double fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    double Rs[9];
    for (int k = 0; k < 9; ++k) Rs[k] = cam[6 + k];
    int64_t n = 0;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            const int64_t p = (int64_t)v * W + u;
            g_depth[p] = 0;
            g_opac[p] = 0;
            for (int k = 0; k < 3; ++k) g_scale[3 * p + k] = 0;
            if (g_quat) for (int k = 0; k < 4; ++k) g_quat[4 * p + k] = 0;
            for (int c = 0; c < C; ++c) g_feat[p * C + c] = 0;
            if (mask && !mask[p]) continue;
            const double ray[3] = {(u - cx) / fx, (v - cy) / fy, 1.0};
            const double *gm = g_mean + 3 * n;
            /* d mean / d z = Rs^T ray */
            double gz = 0;
            for (int i = 0; i < 3; ++i)
                gz += (Rs[0 * 3 + i] * ray[0] + Rs[1 * 3 + i] * ray[1] + Rs[2 * 3 + i] * ray[2]) * gm[i];
            g_depth[p] = gz;
            double w = 1, x = 0, y = 0, zq = 0, nq = 1;
            if (quat) { w = quat[4 * p]; x = quat[4 * p + 1]; y = quat[4 * p + 2]; zq = quat[4 * p + 3]; }
            nq = sqrt(w * w + x * x + y * y + zq * zq);
            w /= nq; x /= nq; y /= nq; zq /= nq;
            const double Rq[3][3] = {
                {1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y)},
                {2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x)},
                {2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)}};
            double Rg[3][3], M[3][3];
            const double s3[3] = {scale[3 * p], scale[3 * p + 1], scale[3 * p + 2]};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    Rg[i][j] = Rs[0 * 3 + i] * Rq[0][j] + Rs[1 * 3 + i] * Rq[1][j] + Rs[2 * 3 + i] * Rq[2][j];
                    M[i][j] = Rg[i][j] * s3[j];
                }
            /* symmetric gradient G of cov = M M^T from the six stored entries */
            const double *gc = g_cov + 6 * n;
            const double G[3][3] = {{gc[0], gc[1] / 2, gc[2] / 2}, {gc[1] / 2, gc[3], gc[4] / 2},
                                    {gc[2] / 2, gc[4] / 2, gc[5]}};
            double gM[3][3];  /* dL/dM = 2 G M */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) gM[i][j] = 2 * (G[i][0] * M[0][j] + G[i][1] * M[1][j] + G[i][2] * M[2][j]);
            for (int j = 0; j < 3; ++j) g_scale[3 * p + j] = gM[0][j] * Rg[0][j] + gM[1][j] * Rg[1][j] + gM[2][j] * Rg[2][j];
            if (g_quat) {
                double gRq[3][3];  /* R_g = Rs^T Rq, dL/dRg[i][j] = gM[i][j] s_j */
                for (int k = 0; k < 3; ++k)
                    for (int j = 0; j < 3; ++j)
                        gRq[k][j] = (Rs[k * 3 + 0] * gM[0][j] + Rs[k * 3 + 1] * gM[1][j] + Rs[k * 3 + 2] * gM[2][j]) * s3[j];
                /* d Rq / d (w, x, y, z) of the normalised quaternion */
                const double gw = 2 * (-zq * gRq[0][1] + y * gRq[0][2] + zq * gRq[1][0] - x * gRq[1][2] - y * gRq[2][0] + x * gRq[2][1]);
                const double gx = 2 * (y * gRq[0][1] + zq * gRq[0][2] + y * gRq[1][0] - 2 * x * gRq[1][1] - w * gRq[1][2]
                                       + zq * gRq[2][0] + w * gRq[2][1] - 2 * x * gRq[2][2]);
                const double gy = 2 * (-2 * y * gRq[0][0] + x * gRq[0][1] + w * gRq[0][2] + x * gRq[1][0] + zq * gRq[1][2]
                                       - w * gRq[2][0] + zq * gRq[2][1] - 2 * y * gRq[2][2]);
                const double gz2 = 2 * (-2 * zq * gRq[0][0] - w * gRq[0][1] + x * gRq[0][2] + w * gRq[1][0] - 2 * zq * gRq[1][1]
                                        + y * gRq[1][2] + x * gRq[2][0] + y * gRq[2][1]);
                /* through q^ = q / |q| */
                const double dot = gw * w + gx * x + gy * y + gz2 * zq;
                g_quat[4 * p] = (gw - w * dot) / nq;
                g_quat[4 * p + 1] = (gx - x * dot) / nq;
                g_quat[4 * p + 2] = (gy - y * dot) / nq;
                g_quat[4 * p + 3] = (gz2 - zq * dot) / nq;
            }
            g_opac[p] = g_op[n];
            for (int c = 0; c < C; ++c) g_feat[p * C + c] = g_ft[n * C + c];
            ++n;
        }
}

/* ------------------------------------------------------------------------
 * Binning: count, exclusive scan, key emission, stable sort, tile ranges.
 * A Gaussian emits one (key, id) pair per tile of its rect, tiles in
 * row-major order, Gaussians in id order; key = tile << 32 | depth bits.
 * The pairs are sorted stably by key, so pairs with equal keys keep
 * ascending Gaussian id.
 * ---------------------------------------------------------------------- */
int64_t orc_scan(int64_t n, const int32_t *ntiles, int64_t *offsets)
{
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) { offsets[i] = acc; acc += ntiles[i]; }
    return acc;
}

void orc_emit(int64_t n, const int32_t *rect, const int64_t *offsets, const uint32_t *dkey,
              int tiles_x, uint64_t *keys, uint32_t *vals)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = offsets[i];
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
                keys[k] = ((uint64_t)(uint32_t)(ty * tiles_x + tx) << 32) | dkey[i];
                vals[k] = (uint32_t)i;
                ++k;
            }
    }
}

/* ------------------------------------------------------------------------
 * Tight binning (an optional variant of the binning above; the paper's
 * rasterizer keeps the whole rect).  A Gaussian can only be blended at a
 * pixel where alpha = o exp(-Q/2) >= alpha_min, Q = d^T conic d, i.e. where
 * Q <= kappa = 2 ln(o / alpha_min).  A tile of the rect is kept when the
 * smallest Q over the rectangle spanned by the tile's pixel centres (clipped
 * to the image) is at most kappa (1 + 2^-10) + 2^-8 -- a margin far above
 * the rounding of any single-precision evaluation of alpha, so that a
 * dropped tile holds no pixel the full rect would have blended.  Rects of
 * more than 32 tiles are kept whole.  Everything here is key mode (strict
 * single precision, in the order written).
 * ------------------------------------------------------------------------ */

/* ln x for finite x >= 1 in key mode, from the mathematics: x = 2^e m with
 * m in [sqrt(1/2), sqrt(2)), ln x = e ln 2 + 2 atanh(t), t = (m - 1)/(m + 1),
 * and atanh(t) = t + t^3/3 + t^5/5 + t^7/7 + t^9/9 + ... (|t| < 0.172, so the
 * terms left out are below 1e-9). */
float orc_key_ln_f32(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    int e = (int)((u >> 23) & 0xffu) - 127;
    uint32_t mb = (u & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > 1.41421354f) {
        m = m * 0.5f;
        e = e + 1;
    }
    const float t = (m - 1.0f) / (m + 1.0f);
    const float t2 = t * t;
    float s = 0.111111111f;
    s = s * t2 + 0.142857143f;
    s = s * t2 + 0.2f;
    s = s * t2 + 0.333333333f;
    s = s * t2 + 1.0f;
    return (float)e * 0.693147182f + 2.0f * (t * s);
}

/* Q = a dx^2 + 2 b dx dy + c dy^2 evaluated as dx (a dx + 2b dy) + (c dy) dy */
static float tight_q(float a, float b2, float c, float dx, float dy)
{
    return dx * (a * dx + b2 * dy) + (c * dy) * dy;
}

static float clampf_(float v, float lo, float hi) { return fminf(hi, fmaxf(lo, v)); }

/* Smallest Q over the rectangle [dx0, dx1] x [dy0, dy1] of offsets from the
 * mean: 0 when the mean lies inside; else the least of the four edge minima
 * (on each edge Q is a parabola, minimised at the clamped vertex). */
static float tight_qmin(float a, float b, float c, float dx0, float dx1, float dy0, float dy1)
{
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return 0.0f;
    const float b2 = 2.0f * b, ra = b / a, rc = b / c;
    float q = INFINITY, d;
    d = clampf_(-(ra * dy0), dx0, dx1); q = fminf(q, tight_q(a, b2, c, d, dy0));
    d = clampf_(-(ra * dy1), dx0, dx1); q = fminf(q, tight_q(a, b2, c, d, dy1));
    d = clampf_(-(rc * dx0), dy0, dy1); q = fminf(q, tight_q(a, b2, c, dx0, d));
    d = clampf_(-(rc * dx1), dy0, dy1); q = fminf(q, tight_q(a, b2, c, dx1, d));
    return q;
}

/* For each Gaussian with ntiles > 0 and a rect of at most 32 tiles: bit
 * (ty - y0) * (x1 - x0) + (tx - x0) of mask[i] is set for a kept tile, and
 * ntiles[i] becomes the number kept (0 culls).  mask[i] = 0xFFFFFFFF for
 * rects kept whole, 0 for culled Gaussians.  opac: the stored opacities;
 * par: params (alpha_min = par[2]); W, H: target size. */
void orc_tight_tiles_f32(int64_t n, const int32_t *rect, const float *mu, const float *conic, const float *opac,
                         const float *par, int W, int H, uint32_t *mask, int32_t *ntiles)
{
    const float amin = par[2];
    for (int64_t i = 0; i < n; ++i) {
        mask[i] = 0u;
        if (ntiles[i] <= 0) continue;
        const int x0 = rect[4 * i], y0 = rect[4 * i + 1], x1 = rect[4 * i + 2], y1 = rect[4 * i + 3];
        const int w = x1 - x0, area = w * (y1 - y0);
        if (area > 32) { mask[i] = 0xFFFFFFFFu; continue; }
        const float ratio = opac[i] / amin;
        uint32_t m = 0u;
        if (ratio >= 1.0f) {
            const float kappa = 2.0f * orc_key_ln_f32(ratio);
            const float thr = kappa * 1.0009765625f + 0.00390625f;
            const float mx = mu[2 * i], my = mu[2 * i + 1];
            const float a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
            for (int ty = y0; ty < y1; ++ty)
                for (int tx = x0; tx < x1; ++tx) {
                    const float px0 = (float)(TILE * tx), py0 = (float)(TILE * ty);
                    const float px1 = (float)(TILE * tx + TILE - 1 < W - 1 ? TILE * tx + TILE - 1 : W - 1);
                    const float py1 = (float)(TILE * ty + TILE - 1 < H - 1 ? TILE * ty + TILE - 1 : H - 1);
                    const float qm = tight_qmin(a, b, c, px0 - mx, px1 - mx, py0 - my, py1 - my);
                    if (qm <= thr) m |= 1u << ((ty - y0) * w + (tx - x0));
                }
        }
        mask[i] = m;
        int cnt = 0;
        for (int k = 0; k < 32; ++k) cnt += (int)((m >> k) & 1u);
        ntiles[i] = cnt;
    }
}

/* Emission with the masks of orc_tight_tiles_f32: the kept tiles of each
 * rect in row-major order (whole rects where mask = 0xFFFFFFFF). */
void orc_emit_masked(int64_t n, const int32_t *rect, const uint32_t *mask, const int64_t *offsets,
                     const uint32_t *dkey, int tiles_x, uint64_t *keys, uint32_t *vals)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = offsets[i];
        const int x0 = rect[4 * i], y0 = rect[4 * i + 1], x1 = rect[4 * i + 2], y1 = rect[4 * i + 3];
        const int w = x1 - x0;
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) {
                const int bit = (ty - y0) * w + (tx - x0);
                if (mask[i] != 0xFFFFFFFFu && (bit >= 32 || !((mask[i] >> bit) & 1u))) continue;
                keys[k] = ((uint64_t)(uint32_t)(ty * tiles_x + tx) << 32) | dkey[i];
                vals[k] = (uint32_t)i;
                ++k;
            }
    }
}

/* Stable bottom-up merge sort of (key, val) on the key alone. */
void orc_sort_pairs(int64_t P, uint64_t *keys, uint32_t *vals)
{
    uint64_t *k2 = (uint64_t *)malloc((size_t)(P > 0 ? P : 1) * sizeof(uint64_t));
    uint32_t *v2 = (uint32_t *)malloc((size_t)(P > 0 ? P : 1) * sizeof(uint32_t));
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int64_t w = 1; w < P; w *= 2) {
        for (int64_t lo = 0; lo < P; lo += 2 * w) {
            int64_t mid = lo + w < P ? lo + w : P;
            int64_t hi = lo + 2 * w < P ? lo + 2 * w : P;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (ka[j] < ka[i]) { kb[o] = ka[j]; vb[o++] = va[j++]; }
                else { kb[o] = ka[i]; vb[o++] = va[i++]; }  /* ties: left run first */
            }
            while (i < mid) { kb[o] = ka[i]; vb[o++] = va[i++]; }
            while (j < hi) { kb[o] = ka[j]; vb[o++] = va[j++]; }
        }
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        memcpy(keys, ka, (size_t)P * sizeof(uint64_t));
        memcpy(vals, va, (size_t)P * sizeof(uint32_t));
    }
    free(k2);
    free(v2);
}

/* range[t] = [first, last+1) of tile t in the sorted keys; [0,0) if empty. */
void orc_ranges(int64_t P, const uint64_t *keys, int n_tiles, uint32_t *ranges)
{
    memset(ranges, 0, (size_t)n_tiles * 2 * sizeof(uint32_t));
    for (int64_t k = 0; k < P; ++k) {
        uint32_t tile = (uint32_t)(keys[k] >> 32);
        if (k == 0 || (uint32_t)(keys[k - 1] >> 32) != tile) ranges[2 * tile] = (uint32_t)k;
        if (k == P - 1 || (uint32_t)(keys[k + 1] >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(k + 1);
    }
}

/* Brute-force list of one tile: every Gaussian whose rect contains the tile,
 * ordered by (depth key, id).  Returns the count. */
int64_t orc_tile_list_bruteforce(int64_t n, const int32_t *rect, const uint32_t *dkey,
                                 int tx, int ty, uint32_t *out)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (tx >= rect[4 * i] && tx < rect[4 * i + 2] && ty >= rect[4 * i + 1] && ty < rect[4 * i + 3])
            out[m++] = (uint32_t)i;
    /* insertion sort by (key, id): tiny inputs only */
    for (int64_t a = 1; a < m; ++a) {
        uint32_t v = out[a];
        int64_t b = a - 1;
        while (b >= 0 && (dkey[out[b]] > dkey[v] || (dkey[out[b]] == dkey[v] && out[b] > v))) {
            out[b + 1] = out[b];
            --b;
        }
        out[b + 1] = v;
    }
    return m;
}

/* ------------------------------------------------------------------------
 * Front-to-back compositing of one pixel (3DGS blending of latent features).
 *
 * For pixel centre p and the tile's list j = start..end-1 in order:
 *   d = p - mu_j,  q = -1/2 (a dx^2 + c dy^2) - b dx dy
 *   q > 0                      -> skip j
 *   alpha = min(alpha_max, o_j e^q)
 *   alpha < alpha_min          -> skip j
 *   T' = T (1 - alpha); T' < t_min -> stop before j
 *   F += f_j alpha T;  T = T'
 * Outputs F, T_final = T, last = 1 + list position of the last blended j
 * (0 if none), A = 1 - T_final.  Background contributes nothing.
 *
 * The paper fixes no precision for these discrete decisions; a decision
 * whose margin is within the given relative tolerance is reported as
 * ambiguous so that a single-precision implementation may take either
 * branch.  `flips` inverts chosen decisions (to produce the alternative
 * outputs), `dec_in` replays recorded decisions (frozen-decision mode for
 * finite differences) and `dec_out` records them.
 * ---------------------------------------------------------------------- */
enum { DEC_Q = 0, DEC_ALPHA = 1, DEC_T = 2 };
enum { REC_SKIP = 0, REC_BLEND = 1, REC_STOP = 2, REC_UNSEEN = 3 };

typedef struct { int64_t k; int type; } decision_t;

typedef struct {
    const double *mu, *conic, *opac, *feat;
    int C;
    double alpha_max, alpha_min, t_min;
    double margin_alpha, margin_t, margin_q;
} comp_in_t;

static int is_flipped(const decision_t *fl, int nfl, int64_t k, int type)
{
    for (int i = 0; i < nfl; ++i)
        if (fl[i].k == k && fl[i].type == type) return 1;
    return 0;
}

static void composite_pixel(const comp_in_t *in, const uint32_t *ids, int64_t start, int64_t end,
                            double px, double py, const decision_t *flips, int nflips,
                            const uint8_t *dec_in, uint8_t *dec_out,
                            double *F, double *Tout, int32_t *last_out,
                            decision_t *amb, int max_amb, int *n_amb)
{
    const int C = in->C;
    double T = 1.0;
    int32_t last = 0;
    int na = 0;
    for (int c = 0; c < C; ++c) F[c] = 0.0;
    if (dec_out)
        for (int64_t k = start; k < end; ++k) dec_out[k - start] = REC_UNSEEN;
    for (int64_t k = start; k < end; ++k) {
        const uint32_t j = ids[k];
        const double dx = px - in->mu[2 * j], dy = py - in->mu[2 * j + 1];
        const double a = in->conic[3 * j], b = in->conic[3 * j + 1], c = in->conic[3 * j + 2];
        const double q = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        const double e = in->opac[j] * exp(q);
        double alpha = e < in->alpha_max ? e : in->alpha_max;
        int blend;
        if (dec_in) {
            uint8_t d = dec_in[k - start];
            if (d == REC_STOP || d == REC_UNSEEN) break;
            blend = (d == REC_BLEND);
        } else {
            double qscale = 0.5 * (fabs(a) * dx * dx + fabs(c) * dy * dy) + fabs(b * dx * dy);
            int skip_q = q > 0;
            if (fabs(q) <= in->margin_q * qscale && qscale > 0) {
                if (na < max_amb) { amb[na].k = k; amb[na].type = DEC_Q; }
                ++na;
            }
            if (is_flipped(flips, nflips, k, DEC_Q)) skip_q = !skip_q;
            if (skip_q) { if (dec_out) dec_out[k - start] = REC_SKIP; continue; }
            int skip_a = alpha < in->alpha_min;
            if (fabs(alpha - in->alpha_min) <= in->margin_alpha * in->alpha_min) {
                if (na < max_amb) { amb[na].k = k; amb[na].type = DEC_ALPHA; }
                ++na;
            }
            if (is_flipped(flips, nflips, k, DEC_ALPHA)) skip_a = !skip_a;
            if (skip_a) { if (dec_out) dec_out[k - start] = REC_SKIP; continue; }
            double Tn = T * (1.0 - alpha);
            int stop = Tn < in->t_min;
            if (fabs(Tn - in->t_min) <= in->margin_t * in->t_min) {
                if (na < max_amb) { amb[na].k = k; amb[na].type = DEC_T; }
                ++na;
            }
            if (is_flipped(flips, nflips, k, DEC_T)) stop = !stop;
            if (stop) { if (dec_out) dec_out[k - start] = REC_STOP; break; }
            blend = 1;
        }
        if (!blend) { if (dec_out) dec_out[k - start] = REC_SKIP; continue; }
        const double w = alpha * T;
        const double *f = in->feat + (int64_t)j * C;
        for (int ch = 0; ch < C; ++ch) F[ch] += f[ch] * w;
        T = T * (1.0 - alpha);
        last = (int32_t)(k - start + 1);
        if (dec_out) dec_out[k - start] = REC_BLEND;
    }
    *Tout = T;
    *last_out = last;
    if (n_amb) *n_amb = na;
}

#define MAX_AMB 8

/* Composite every pixel of the listed tiles (all tiles if tile_list is
 * NULL).  flags[p] = number of ambiguous decisions of pixel p (saturating
 * at 255).  dec_in/dec_out (optional) hold 256*P bytes laid out per tile:
 * tile t, pixel slot s (row-major in the tile), list position k at
 * 256*start_t + s*(end_t-start_t) + (k-start_t). */
void orc_composite(int64_t n, const double *mu, const double *conic, const double *opac,
                   const double *feat, int C, int W, int H, const uint32_t *ranges,
                   const uint32_t *ids, const float *par, const double *margins,
                   int n_list, const int32_t *tile_list,
                   double *F, double *A, double *Tfin, int32_t *last, uint8_t *flags,
                   const uint8_t *dec_in, uint8_t *dec_out)
{
    (void)n;
    comp_in_t in = {mu, conic, opac, feat, C, par[1], par[2], par[3],
                    margins ? margins[0] : 0.0, margins ? margins[1] : 0.0, margins ? margins[2] : 0.0};
    const int tiles_x = (W + TILE - 1) / TILE, tiles_y = (H + TILE - 1) / TILE;
    const int nt = tile_list ? n_list : tiles_x * tiles_y;
    const int64_t HW = (int64_t)W * H;
#pragma omp parallel
    {
        double *f = (double *)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
        decision_t amb[MAX_AMB];
#pragma omp for schedule(dynamic, 1)
        for (int it = 0; it < nt; ++it) {
            const int tile = tile_list ? tile_list[it] : it;
            const int tx = tile % tiles_x, ty = tile / tiles_x;
            const int64_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
            for (int s = 0; s < TILE * TILE; ++s) {
                const int x = tx * TILE + s % TILE, y = ty * TILE + s / TILE;
                if (x >= W || y >= H) continue;
                const int64_t pix = (int64_t)y * W + x;
                const int64_t doff = 256 * start + (int64_t)s * (end - start);
                double T;
                int32_t lst;
                int na = 0;
                composite_pixel(&in, ids, start, end, (double)x, (double)y, NULL, 0,
                                dec_in ? dec_in + doff : NULL, dec_out ? dec_out + doff : NULL,
                                f, &T, &lst, amb, MAX_AMB, &na);
                for (int c = 0; c < C; ++c) F[c * HW + pix] = f[c];
                A[pix] = 1.0 - T;
                if (Tfin) Tfin[pix] = T;
                if (last) last[pix] = lst;
                if (flags) flags[pix] = (uint8_t)(na > 255 ? 255 : na);
            }
        }
        free(f);
    }
    (void)tiles_y;
}

/* Alternative outputs of one pixel whose decisions are ambiguous: every
 * non-empty subset of its (at most max_flip) ambiguous decisions is
 * inverted in turn.  Writes n_alt x (C+1) values (F then A) and returns
 * n_alt, or -1 if the pixel has more ambiguous decisions than max_flip. */
int orc_pixel_alternatives(const double *mu, const double *conic, const double *opac,
                           const double *feat, int C, int W, int H, const uint32_t *ranges,
                           const uint32_t *ids, const float *par, const double *margins,
                           int x, int y, int max_flip, double *out)
{
    (void)H;
    comp_in_t in = {mu, conic, opac, feat, C, par[1], par[2], par[3], margins[0], margins[1], margins[2]};
    const int tiles_x = (W + TILE - 1) / TILE;
    const int tile = (y / TILE) * tiles_x + x / TILE;
    const int64_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    decision_t amb[MAX_AMB];
    int na = 0;
    double *f = (double *)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    double T;
    int32_t lst;
    composite_pixel(&in, ids, start, end, x, y, NULL, 0, NULL, NULL, f, &T, &lst, amb, MAX_AMB, &na);
    if (na > max_flip || na > MAX_AMB) { free(f); return -1; }
    int n_alt = 0;
    for (int mask = 1; mask < (1 << na); ++mask) {
        decision_t fl[MAX_AMB];
        int nfl = 0;
        for (int b = 0; b < na; ++b)
            if (mask & (1 << b)) fl[nfl++] = amb[b];
        composite_pixel(&in, ids, start, end, x, y, fl, nfl, NULL, NULL, f, &T, &lst, NULL, 0, NULL);
        for (int c = 0; c < C; ++c) out[n_alt * (C + 1) + c] = f[c];
        out[n_alt * (C + 1) + C] = 1.0 - T;
        ++n_alt;
    }
    free(f);
    return n_alt;
}

/* ------------------------------------------------------------------------
 * Adjoint of the compositing (the rasterizer is differentiated end to end
 * in the paper, Sec. 4.2).  With g = dL/dF(p), gA = dL/dA(p), T_j the
 * transmittance in front of the blended Gaussian j and
 * S_j = sum over blended k behind j of alpha_k T_k <f_k, g>:
 *   dL/df_j     += alpha_j T_j g
 *   dL/dalpha_j  = T_j <f_j, g> - S_j / (1 - alpha_j) + gA T_final / (1 - alpha_j)
 * and through alpha = o e^q (no gradient where alpha was clamped to
 * alpha_max), q = -1/2 (a dx^2 + c dy^2) - b dx dy, d = p - mu:
 *   dL/do  += e^q dL/dalpha;   dL/dq = alpha dL/dalpha
 *   dL/d(a,b,c) += dL/dq (-dx^2/2, -dx dy, -dy^2/2)
 *   dL/dmu      += dL/dq (a dx + b dy, b dx + c dy)
 * The decisions are the forward's (ambiguity margins do not apply here).
 * Single-threaded; gradients are accumulated in double.
 * ---------------------------------------------------------------------- */
void orc_backward(int64_t n, const double *mu, const double *conic, const double *opac,
                  const double *feat, int C, int W, int H, const uint32_t *ranges,
                  const uint32_t *ids, const float *par, const double *dF, const double *dA,
                  double *d_mu, double *d_conic, double *d_opac, double *d_feat)
{
    (void)n;
    const double alpha_max = par[1], alpha_min = par[2], t_min = par[3];
    const int tiles_x = (W + TILE - 1) / TILE, tiles_y = (H + TILE - 1) / TILE;
    const int64_t HW = (int64_t)W * H;
    int64_t maxlen = 1;
    for (int t = 0; t < tiles_x * tiles_y; ++t)
        if ((int64_t)ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
    int64_t *lk = (int64_t *)malloc(sizeof(int64_t) * (size_t)maxlen);
    double *la = (double *)malloc(sizeof(double) * (size_t)maxlen);
    double *lT = (double *)malloc(sizeof(double) * (size_t)maxlen);
    double *le = (double *)malloc(sizeof(double) * (size_t)maxlen);
    int *lc = (int *)malloc(sizeof(int) * (size_t)maxlen);
    double *g = (double *)malloc(sizeof(double) * (size_t)(C > 0 ? C : 1));
    for (int tile = 0; tile < tiles_x * tiles_y; ++tile) {
        const int tx = tile % tiles_x, ty = tile / tiles_x;
        const int64_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
        for (int s = 0; s < TILE * TILE; ++s) {
            const int x = tx * TILE + s % TILE, y = ty * TILE + s / TILE;
            if (x >= W || y >= H) continue;
            const int64_t pix = (int64_t)y * W + x;
            /* forward pass: record the blended Gaussians */
            int64_t m = 0;
            double T = 1.0;
            for (int64_t k = start; k < end; ++k) {
                const uint32_t j = ids[k];
                const double dx = x - mu[2 * j], dy = y - mu[2 * j + 1];
                const double q = -0.5 * (conic[3 * j] * dx * dx + conic[3 * j + 2] * dy * dy) - conic[3 * j + 1] * dx * dy;
                if (q > 0) continue;
                const double e = opac[j] * exp(q);
                const double alpha = e < alpha_max ? e : alpha_max;
                if (alpha < alpha_min) continue;
                const double Tn = T * (1.0 - alpha);
                if (Tn < t_min) break;
                lk[m] = k; la[m] = alpha; lT[m] = T; le[m] = exp(q); lc[m] = !(e < alpha_max);
                ++m;
                T = Tn;
            }
            const double Tfinal = T;
            for (int c = 0; c < C; ++c) g[c] = dF[c * HW + pix];
            const double gA = dA ? dA[pix] : 0.0;
            double S = 0.0;
            for (int64_t r = m - 1; r >= 0; --r) {
                const uint32_t j = ids[lk[r]];
                const double *f = feat + (int64_t)j * C;
                double fg = 0.0;
                for (int c = 0; c < C; ++c) fg += f[c] * g[c];
                const double alpha = la[r], Tj = lT[r];
                for (int c = 0; c < C; ++c) d_feat[(int64_t)j * C + c] += alpha * Tj * g[c];
                const double dalpha = Tj * fg - S / (1.0 - alpha) + gA * Tfinal / (1.0 - alpha);
                S += alpha * Tj * fg;
                if (lc[r]) continue;
                const double dx = x - mu[2 * j], dy = y - mu[2 * j + 1];
                const double a = conic[3 * j], b = conic[3 * j + 1], c = conic[3 * j + 2];
                d_opac[j] += le[r] * dalpha;
                const double dq = alpha * dalpha;
                d_conic[3 * j] += dq * (-0.5 * dx * dx);
                d_conic[3 * j + 1] += dq * (-dx * dy);
                d_conic[3 * j + 2] += dq * (-0.5 * dy * dy);
                d_mu[2 * j] += dq * (a * dx + b * dy);
                d_mu[2 * j + 1] += dq * (b * dx + c * dy);
            }
        }
    }
    free(lk); free(la); free(lT); free(le); free(lc); free(g);
}
