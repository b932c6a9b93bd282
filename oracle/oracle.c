/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the per-frame hot
 * path of "Real-Time Polygonal Semantic Mapping for Humanoid Robot Stair
 * Climbing" (arXiv 2411.01919): anisotropic diffusion of the depth image,
 * back-projection + normal image, and sequential multi-plane RANSAC.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only the test suite, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant table with the CUDA
 * implementation.
 *
 * Precision: FP64 throughout, except where a floating-point result decides an
 * integer (which points are inliers, hence the RANSAC counts, the argmax, the
 * inlier labels).  Those decisions are taken in FP32, the precision the
 * method's GPU scoring runs in, with every operation spelled out below
 * (IEEE-754 round-to-nearest, no contraction except the explicit fmaf calls).
 * Compile with -ffp-contract=off.
 *
 * Every function cites the passage of the paper it follows.  Readings where
 * the paper is silent or garbled are stated at the function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Depth decoding (Sec. III-A / III-B: the sensor delivers a depth image).   */
/* ------------------------------------------------------------------------ */

/* IEEE 754 binary16 -> double, from the format's definition:
 * 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
double or_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int expo = (h >> 10) & 0x1f;
    int frac = h & 0x3ff;
    double v;
    if (expo == 0)
        v = ldexp((double)frac, -24);                 /* subnormal: frac * 2^-14 * 2^-10 */
    else if (expo == 31)
        v = frac ? NAN : INFINITY;
    else
        v = ldexp((double)(frac + 1024), expo - 25);  /* (1 + frac/1024) * 2^(e-15) */
    return sign ? -v : v;
}

/* dtype: 0 = u16 in units of depth_scale metres, 1 = f16 metres, 2 = f32 metres.
 * A value that is zero, negative or not finite marks a hole; holes decode to 0. */
int or_decode(const void *src, int dtype, int w, int h, long pitch_bytes,
              double depth_scale, double *out)
{
    for (int v = 0; v < h; ++v) {
        const unsigned char *row = (const unsigned char *)src + (long)v * pitch_bytes;
        for (int u = 0; u < w; ++u) {
            double z;
            if (dtype == 0) {
                uint16_t q;
                memcpy(&q, row + 2 * (long)u, 2);
                z = (double)q * depth_scale;
            } else if (dtype == 1) {
                uint16_t q;
                memcpy(&q, row + 2 * (long)u, 2);
                z = or_half_to_double(q);
            } else if (dtype == 2) {
                float f;
                memcpy(&f, row + 4 * (long)u, 4);
                z = (double)f;
            } else {
                return -1;
            }
            if (!(z > 0.0) || !isfinite(z))
                z = 0.0;
            out[(long)v * w + u] = z;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Anisotropic diffusion: Eq. 1 and Alg. 1 (the smoothing loop).             */
/* ------------------------------------------------------------------------ */

/* Value the stencil sees for neighbour (qu, qv) of pixel p.  Reading of the
 * paper's silence on borders and holes: a neighbour outside the image or on a
 * hole is replaced by the centre value I_p, so no flux crosses the image border
 * or a hole (zero-flux / Neumann boundary). */
static double ghost(const double *I, const unsigned char *valid, int w, int h,
                    int qu, int qv, double Ip)
{
    if (qu < 0 || qu >= w || qv < 0 || qv >= h)
        return Ip;
    long q = (long)qv * w + qu;
    return valid[q] ? I[q] : Ip;
}

/* mode 0 (PM4): the 4-neighbour discretisation of Eq. 1 with the exponential
 *   conductance g(x) = exp(-(x/K)^2) evaluated on each neighbour difference:
 *     I'_p = I_p + lambda * sum_q g(J_q - I_p) (J_q - I_p).
 * mode 1 (ALG1): Alg. 1 read literally: one conductance per pixel from the
 *   central-difference gradient magnitude, times the 4-neighbour Laplacian:
 *     |grad I_p| = sqrt(((J_E - J_W)/2)^2 + ((J_S - J_N)/2)^2),
 *     c_p = exp(-(|grad I_p| / K)^2),  I'_p = I_p + lambda c_p sum_q (J_q - I_p).
 * Jacobi iteration (all pixels updated from the previous iterate, "for each
 * pixel ... parallel").  Holes keep the value 0.  Requires 0 < lambda <= 1/4. */
int or_diffuse(const double *in, double *out, int w, int h, int iters,
               double lambda, double K, int mode)
{
    long n = (long)w * h;
    if (w <= 0 || h <= 0 || iters < 0 || !(lambda > 0.0) || lambda > 0.25 || !(K > 0.0))
        return -1;
    unsigned char *valid = (unsigned char *)malloc((size_t)n);
    double *cur = (double *)malloc((size_t)n * sizeof(double));
    double *nxt = (double *)malloc((size_t)n * sizeof(double));
    if (!valid || !cur || !nxt) {
        free(valid); free(cur); free(nxt);
        return -2;
    }
    for (long i = 0; i < n; ++i) {
        valid[i] = (in[i] > 0.0) && isfinite(in[i]);
        cur[i] = valid[i] ? in[i] : 0.0;
    }
    for (int it = 0; it < iters; ++it) {
        for (int v = 0; v < h; ++v) {
            for (int u = 0; u < w; ++u) {
                long p = (long)v * w + u;
                if (!valid[p]) {
                    nxt[p] = 0.0;
                    continue;
                }
                double Ip = cur[p];
                double JN = ghost(cur, valid, w, h, u, v - 1, Ip);
                double JS = ghost(cur, valid, w, h, u, v + 1, Ip);
                double JW = ghost(cur, valid, w, h, u - 1, v, Ip);
                double JE = ghost(cur, valid, w, h, u + 1, v, Ip);
                if (mode == 0) {
                    double J[4] = {JN, JS, JW, JE};
                    double s = 0.0;
                    for (int k = 0; k < 4; ++k) {
                        double x = J[k] - Ip;
                        double g = exp(-(x / K) * (x / K));
                        s += g * x;
                    }
                    nxt[p] = Ip + lambda * s;
                } else {
                    double gx = (JE - JW) / 2.0;
                    double gy = (JS - JN) / 2.0;
                    double grad = sqrt(gx * gx + gy * gy);
                    double c = exp(-(grad / K) * (grad / K));
                    double lap = (JN - Ip) + (JS - Ip) + (JW - Ip) + (JE - Ip);
                    nxt[p] = Ip + lambda * c * lap;
                }
            }
        }
        double *t = cur; cur = nxt; nxt = t;
    }
    memcpy(out, cur, (size_t)n * sizeof(double));
    free(valid); free(cur); free(nxt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Back-projection and normals: Alg. 1 (normal loop), Eq. 2, Alg. 2.          */
/* ------------------------------------------------------------------------ */

/* Reading of Eq. 2 (dimensionally garbled as printed): the normal at a pixel
 * is the exact surface normal of the back-projected depth map,
 *   P(u,v) = z(u,v) ((u - cx)/fx, (v - cy)/fy, 1),
 *   n = normalize(t_u x t_v), oriented so that n . P(u,v) < 0 (towards the camera),
 * with t_u, t_v the horizontal and vertical point differences:
 *   stencil 0 (central): t_u = P(u+1,v) - P(u-1,v), t_v = P(u,v+1) - P(u,v-1);
 *   stencil 1 (Sobel):   the same differences weighted (1,2,1) across the
 *                        perpendicular direction, as the Sobel operator does.
 * A normal is invalid on the one-pixel border, next to a hole, or when the
 * cross product vanishes.
 * Outputs: P and N in SoA layout [3][h*w]; valid bit 0 = depth valid,
 * bit 1 = normal valid.  Holes get P = N = 0. */
int or_normals(const double *z, int w, int h, double fx, double fy, double cx, double cy,
               int stencil, double *P, double *N, unsigned char *valid)
{
    long n = (long)w * h;
    if (w <= 0 || h <= 0 || !(fx > 0) || !(fy > 0) || (stencil != 0 && stencil != 1))
        return -1;
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u) {
            long p = (long)v * w + u;
            double zz = z[p];
            int ok = (zz > 0.0) && isfinite(zz);
            P[p] = ok ? zz * ((u - cx) / fx) : 0.0;
            P[n + p] = ok ? zz * ((v - cy) / fy) : 0.0;
            P[2 * n + p] = ok ? zz : 0.0;
            valid[p] = (unsigned char)(ok ? 1 : 0);
            N[p] = N[n + p] = N[2 * n + p] = 0.0;
        }
    for (int v = 1; v < h - 1; ++v)
        for (int u = 1; u < w - 1; ++u) {
            long p = (long)v * w + u;
            double tu[3] = {0, 0, 0}, tv[3] = {0, 0, 0};
            int ok = 1;
            if (stencil == 0) {
                long a = p + 1, b = p - 1, c = p + w, d = p - w;
                ok = valid[p] && valid[a] && valid[b] && valid[c] && valid[d];
                for (int k = 0; k < 3; ++k) {
                    tu[k] = P[k * n + a] - P[k * n + b];
                    tv[k] = P[k * n + c] - P[k * n + d];
                }
            } else {
                static const double wt[3] = {1.0, 2.0, 1.0};
                for (int dv = -1; dv <= 1; ++dv)
                    for (int du = -1; du <= 1; ++du)
                        ok = ok && valid[p + (long)dv * w + du];
                for (int j = -1; j <= 1; ++j) {
                    long r = p + (long)j * w;   /* row v+j, for t_u */
                    long c = p + j;             /* column u+j, for t_v */
                    for (int k = 0; k < 3; ++k) {
                        tu[k] += wt[j + 1] * (P[k * n + r + 1] - P[k * n + r - 1]);
                        tv[k] += wt[j + 1] * (P[k * n + c + w] - P[k * n + c - w]);
                    }
                }
            }
            if (!ok)
                continue;
            double c0 = tu[1] * tv[2] - tu[2] * tv[1];
            double c1 = tu[2] * tv[0] - tu[0] * tv[2];
            double c2 = tu[0] * tv[1] - tu[1] * tv[0];
            double len = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
            if (!(len > 0.0))
                continue;
            c0 /= len; c1 /= len; c2 /= len;
            if (c0 * P[p] + c1 * P[n + p] + c2 * P[2 * n + p] > 0.0) {
                c0 = -c0; c1 = -c1; c2 = -c2;
            }
            N[p] = c0; N[n + p] = c1; N[2 * n + p] = c2;
            valid[p] |= 2;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11).  Source of the    */
/* "random subset of 3 points" of Alg. 2.                                    */
/* ------------------------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* One Philox4xW bijection with `rounds` rounds, parameterised by the round
 * multipliers m0, m1 and the key increments (Weyl constants) w0, w1.  Each
 * round: (hi0, lo0) = m0 * c0, (hi1, lo1) = m1 * c2,
 *        c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is bumped. */
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], int rounds,
                   uint64_t m0, uint64_t m1, uint64_t w0, uint64_t w1, uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < rounds; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(m0, c0, &hi0, &lo0);
        mulhilo64(m1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += w0; k1 += w1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The published Philox4x64 constants. */
#define OR_PHILOX_M0 0xD2E7470EE14C6C93ULL
#define OR_PHILOX_M1 0xCA5A826395121157ULL
#define OR_PHILOX_W0 0x9E3779B97F4A7C15ULL   /* golden ratio */
#define OR_PHILOX_W1 0xBB67AE8584CAA73BULL   /* sqrt(3) - 1 */

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    or_philox4x64(ctr, key, 10, OR_PHILOX_M0, OR_PHILOX_M1, OR_PHILOX_W0, OR_PHILOX_W1, out);
}

/* ------------------------------------------------------------------------ */
/* 3x3 symmetric eigen-decomposition by cyclic Jacobi rotations              */
/* (Golub & Van Loan, Matrix Computations, Sec. 8.5).  A is row-major;       */
/* evals ascending; evecs row-major with eigenvector k in column k.          */
/* ------------------------------------------------------------------------ */
void or_eig3(const double A_in[9], double evals[3], double evecs[9])
{
    double A[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = A_in[3 * i + j];
            V[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-40 * dia)
            break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0)
                    continue;
                double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < 3; ++k) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (A[idx[j]][idx[j]] < A[idx[i]][idx[i]]) {
                int t = idx[i]; idx[i] = idx[j]; idx[j] = t;
            }
    for (int k = 0; k < 3; ++k) {
        evals[k] = A[idx[k]][idx[k]];
        for (int i = 0; i < 3; ++i)
            evecs[3 * i + k] = V[i][idx[k]];
    }
}

/* ------------------------------------------------------------------------ */
/* Multi-plane RANSAC: Eq. 3 and Alg. 2, in whole-frame sequential form.     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double n[3];
    double d;
    int n_inliers;     /* inliers of the winning hypothesis (labelled) */
    int n_refit;       /* points used in the refit */
    double rms;        /* RMS distance of the refit points to the refit plane */
    int hyp_index;     /* winning hypothesis */
    int band;          /* candidates whose FP64 residual lies within 1e-6 m of the threshold */
} or_plane;

/* The FP32 hypothesis plane of Alg. 2 ("fit plane model to these points"):
 * n = (p1 - p0) x (p2 - p0), normalised, d = -n . p0, every step one IEEE
 * FP32 operation in the order written.  Degenerate (returns 0) when
 * |n|^2 <= 1e-18 m^4, i.e. |n| <= 1e-9 m^2, which includes repeated indices. */
static int hyp_plane_f32(const float p0[3], const float p1[3], const float p2[3], float out[4])
{
    float e1x = p1[0] - p0[0], e1y = p1[1] - p0[1], e1z = p1[2] - p0[2];
    float e2x = p2[0] - p0[0], e2y = p2[1] - p0[1], e2z = p2[2] - p0[2];
    float a, b;
    a = e1y * e2z; b = e1z * e2y; float nx = a - b;
    a = e1z * e2x; b = e1x * e2z; float ny = a - b;
    a = e1x * e2y; b = e1y * e2x; float nz = a - b;
    float xx = nx * nx, yy = ny * ny, zz = nz * nz;
    float nn = xx + yy;
    nn = nn + zz;
    if (!(nn > 1e-18f))
        return 0;
    float s = sqrtf(nn);
    nx = nx / s; ny = ny / s; nz = nz / s;
    float t0 = nx * p0[0], t1 = ny * p0[1], t2 = nz * p0[2];
    float dot = t0 + t1;
    dot = dot + t2;
    out[0] = nx; out[1] = ny; out[2] = nz; out[3] = -dot;
    return 1;
}

/* The FP32 inlier decision of Alg. 2 ("d < threshold"): the residual
 * r = n.p + d evaluated as fma(nz, pz, fma(ny, py, fma(nx, px, d))), and the
 * point is an inlier when r*r < thr^2 with the square taken exactly inside one
 * fused multiply-add: fma(r, r, -thr2) < 0, thr2 = thr*thr rounded to FP32. */
static int is_inlier_f32(const float pl[4], float px, float py, float pz, float thr2)
{
    float r = fmaf(pl[0], px, pl[3]);
    r = fmaf(pl[1], py, r);
    r = fmaf(pl[2], pz, r);
    return fmaf(r, r, -thr2) < 0.0f;
}

/* key = (seed, 0); counter = (h, round, frame_idx, 0); the three indices are
 * i_j = floor(w_j * M / 2^64) for the first three output words. */
static void draw_indices(uint64_t seed, uint64_t frame_idx, int round, int hyp, uint64_t M, uint64_t idx[3])
{
    uint64_t key[2] = {seed, 0};
    uint64_t ctr[4] = {(uint64_t)hyp, (uint64_t)round, frame_idx, 0};
    uint64_t w[4];
    or_philox4x64_10(ctr, key, w);
    for (int j = 0; j < 3; ++j) {
        unsigned __int128 prod = (unsigned __int128)w[j] * M;
        idx[j] = (uint64_t)(prod >> 64);
    }
}

/* Sequential multi-plane RANSAC over one frame (Alg. 2 applied to the whole
 * frame, plane after plane, as the paper's host loop does per polygon).
 *   P, N: SoA [3][w*h] FP32 points and normals (N may be NULL: no refit gate).
 *   valid: bit 0 = point valid, bit 1 = normal valid.
 * Round r:
 *   candidates = valid points not yet labelled (M of them), enumerated in
 *     strips of two rows (rows 2s and 2s + 1; one row if h is odd and it is
 *     the last), each strip column by column, the upper pixel first;
 *   hypothesis h < H: three Philox indices -> FP32 plane (hyp_plane_f32);
 *   count_h = #inliers (is_inlier_f32); degenerate hypotheses count -1;
 *   winner = maximum count, ties to the lowest h ("best model" of Alg. 2 with
 *   the inlier count as the score);
 *   stop without a plane if the winner has fewer than min_inliers inliers;
 *   label the winner's inliers with r;
 *   refit in FP64 by PCA over the inliers whose normal is valid and within
 *   gate_deg of the hypothesis normal, decided in FP32 as |n . h| >= cos of
 *   the gate angle (all inliers if fewer than 3 pass):
 *   n = eigenvector of the smallest covariance eigenvalue, d = -n . centroid,
 *   oriented towards the camera (d > 0).
 * Outputs: planes[max_planes], labels[w*h] (-1 = none), optional per-round
 * counts[max_planes * H] and the number of rounds run.  Returns the number of
 * planes, or -1 on bad arguments, -2 on allocation failure. */
int or_ransac(const float *P, const float *N, const unsigned char *valid, int w, int h,
              int H, float thr, int max_planes, int min_inliers, uint64_t seed,
              double gate_deg, uint64_t frame_idx,
              or_plane *planes, short *labels, int *counts_out)
{
    long n = (long)w * h;
    if (w <= 0 || h <= 0 || H <= 0 || !(thr > 0.0f) || max_planes <= 0 || max_planes > 32767)
        return -1;
    long *cand = (long *)malloc((size_t)n * sizeof(long));
    int *counts = (int *)malloc((size_t)H * sizeof(int));
    float (*hyp)[4] = (float (*)[4])malloc((size_t)H * sizeof(float[4]));
    unsigned char *inl = (unsigned char *)malloc((size_t)n);
    if (!cand || !counts || !hyp || !inl) {
        free(cand); free(counts); free(hyp); free(inl);
        return -2;
    }
    float thr2 = thr * thr;
    /* the refit gate decides which inliers the refit uses (an integer set),
     * so it is taken in FP32 with its operations spelled out, like the
     * inlier test: cos of the gate angle rounded once to FP32, the dot
     * product of the FP32 normals as fma(nz, hz, fma(ny, hy, nx * hx)) */
    float cos_gate = (float)cos(gate_deg * M_PI / 180.0);
    for (long i = 0; i < n; ++i)
        labels[i] = -1;
    int n_planes = 0;
    for (int r = 0; r < max_planes; ++r) {
        long M = 0;
        for (int y0 = 0; y0 < h; y0 += 2)          /* strips of two rows */
            for (int x = 0; x < w; ++x)              /* column by column */
                for (int y = y0; y < y0 + 2 && y < h; ++y) {
                    long i = (long)y * w + x;
                    if ((valid[i] & 1) && labels[i] < 0)
                        cand[M++] = i;
                }
        for (int hh = 0; hh < H; ++hh) {
            counts[hh] = -1;
            if (M == 0)
                continue;
            uint64_t idx[3];
            draw_indices(seed, frame_idx, r, hh, (uint64_t)M, idx);
            float p[3][3];
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    p[j][k] = P[k * n + cand[idx[j]]];
            if (!hyp_plane_f32(p[0], p[1], p[2], hyp[hh]))
                continue;
            int c = 0;
            for (long m = 0; m < M; ++m) {
                long i = cand[m];
                c += is_inlier_f32(hyp[hh], P[i], P[n + i], P[2 * n + i], thr2);
            }
            counts[hh] = c;
        }
        if (counts_out)
            memcpy(counts_out + (long)r * H, counts, (size_t)H * sizeof(int));
        int best = 0;
        for (int hh = 1; hh < H; ++hh)
            if (counts[hh] > counts[best])
                best = hh;
        if (M == 0 || counts[best] < min_inliers || counts[best] < 3)
            break;

        /* label the winner's inliers; FP64 residual band for reporting */
        const float *pl = hyp[best];
        uint64_t idx[3];
        draw_indices(seed, frame_idx, r, best, (uint64_t)M, idx);
        double q[3][3];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                q[j][k] = (double)P[k * n + cand[idx[j]]];
        double e1[3] = {q[1][0] - q[0][0], q[1][1] - q[0][1], q[1][2] - q[0][2]};
        double e2[3] = {q[2][0] - q[0][0], q[2][1] - q[0][1], q[2][2] - q[0][2]};
        double m64[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                         e1[0] * e2[1] - e1[1] * e2[0]};
        double l64 = sqrt(m64[0] * m64[0] + m64[1] * m64[1] + m64[2] * m64[2]);
        for (int k = 0; k < 3; ++k)
            m64[k] /= l64;
        double d64 = -(m64[0] * q[0][0] + m64[1] * q[0][1] + m64[2] * q[0][2]);
        int n_in = 0, band = 0, n_gate = 0;
        for (long m = 0; m < M; ++m) {
            long i = cand[m];
            double r64 = m64[0] * P[i] + m64[1] * P[n + i] + m64[2] * P[2 * n + i] + d64;
            if (fabs(fabs(r64) - (double)thr) <= 1e-6)
                band++;
            inl[m] = 0;
            if (is_inlier_f32(pl, P[i], P[n + i], P[2 * n + i], thr2)) {
                labels[i] = (short)r;
                n_in++;
                int gated = 0;
                if (N && (valid[i] & 2)) {
                    float dot = fmaf(N[2 * n + i], pl[2], fmaf(N[n + i], pl[1], N[i] * pl[0]));
                    gated = fabsf(dot) >= cos_gate;
                }
                inl[m] = (unsigned char)(1 + gated);
                n_gate += gated;
            }
        }
        int use_gate = n_gate >= 3;

        /* FP64 refit: mean, covariance, smallest eigenvector */
        double c[3] = {0, 0, 0};
        int cnt = 0;
        for (long m = 0; m < M; ++m) {
            if (!inl[m] || (use_gate && inl[m] != 2))
                continue;
            long i = cand[m];
            c[0] += P[i]; c[1] += P[n + i]; c[2] += P[2 * n + i];
            cnt++;
        }
        for (int k = 0; k < 3; ++k)
            c[k] /= cnt;
        double C[9] = {0};
        for (long m = 0; m < M; ++m) {
            if (!inl[m] || (use_gate && inl[m] != 2))
                continue;
            long i = cand[m];
            double x[3] = {P[i] - c[0], P[n + i] - c[1], P[2 * n + i] - c[2]};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    C[3 * a + b] += x[a] * x[b];
        }
        for (int k = 0; k < 9; ++k)
            C[k] /= cnt;
        double ev[3], V[9];
        or_eig3(C, ev, V);
        double nn[3] = {V[0], V[3], V[6]};
        double ln = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int k = 0; k < 3; ++k)
            nn[k] /= ln;
        double d = -(nn[0] * c[0] + nn[1] * c[1] + nn[2] * c[2]);
        if (d < 0) {
            for (int k = 0; k < 3; ++k)
                nn[k] = -nn[k];
            d = -d;
        }
        double ss = 0.0;
        for (long m = 0; m < M; ++m) {
            if (!inl[m] || (use_gate && inl[m] != 2))
                continue;
            long i = cand[m];
            double e = nn[0] * P[i] + nn[1] * P[n + i] + nn[2] * P[2 * n + i] + d;
            ss += e * e;
        }
        or_plane *o = &planes[n_planes++];
        for (int k = 0; k < 3; ++k)
            o->n[k] = nn[k];
        o->d = d;
        o->n_inliers = n_in;
        o->n_refit = cnt;
        o->rms = sqrt(ss / cnt);
        o->hyp_index = best;
        o->band = band;
    }
    free(cand); free(counts); free(hyp); free(inl);
    return n_planes;
}

/* ------------------------------------------------------------------------ */
/* Per-region RANSAC in the literal form of Alg. 2 (one model per polygon). */
/* ------------------------------------------------------------------------ */

typedef struct {
    double n[3];
    double d;
    unsigned long long error;   /* sum of distances in units of 2^-32 m */
    int inliers;
    int total;
    int accepted;
    int hyp_index;
} or_region_plane;

#define OR_REGION_TRIES 64

/* The point sample of Alg. 2 ("select random subset of 3 points") for
 * region r: for sample j in {0, 1, 2}, attempt a = 0..63 draws
 *   Philox4x64-10(key = (seed, 1), counter = (h, r, frame_idx, 64 j + a))
 * and takes the pixel (u0 + floor(w0 * bw / 2^64), v0 + floor(w1 * bh / 2^64))
 * of the region's bounding box [u0, u0 + bw) x [v0, v0 + bh); the first
 * attempt that lands on a valid point of the region is the sample (uniform
 * over the region's points, by rejection).  Returns 0 if some sample found no
 * point in 64 attempts (then the hypothesis is degenerate). */
static int region_sample(uint64_t seed, uint64_t frame_idx, int r, int h, int u0, int v0, int bw,
                         int bh, int w, const int *regions, const unsigned char *valid,
                         long out[3])
{
    for (int j = 0; j < 3; ++j) {
        out[j] = -1;
        for (int a = 0; a < OR_REGION_TRIES; ++a) {
            uint64_t key[2] = {seed, 1};
            uint64_t ctr[4] = {(uint64_t)h, (uint64_t)r, frame_idx, (uint64_t)(64 * j + a)};
            uint64_t wd[4];
            or_philox4x64_10(ctr, key, wd);
            int u = u0 + (int)(((unsigned __int128)wd[0] * (uint64_t)bw) >> 64);
            int v = v0 + (int)(((unsigned __int128)wd[1] * (uint64_t)bh) >> 64);
            long p = (long)v * w + u;
            if ((valid[p] & 1) && regions[p] == r) {
                out[j] = p;
                break;
            }
        }
        if (out[j] < 0)
            return 0;
    }
    return 1;
}

/* Alg. 2 for every region r in [0, R) of one frame (regions[p] = region of
 * pixel p, < 0 or >= R: none): for each of H hypotheses, the FP32 plane
 * through its three samples (hyp_plane_f32) and
 *   error_h = sum over the region's valid points of d_i,
 *   d_i = |r_i| with r_i the FP32 residual of is_inlier_f32, truncated to a
 *         multiple of 2^-32 m (d_i * 2^32 is exact in FP32) and summed exactly
 *         in 64-bit integers;
 *   inliers_h = #{ i : fma(r_i, r_i, -thr^2) < 0 }   (Alg. 2 "d < threshold");
 * the winner minimises error_h (ties: lowest h; degenerate hypotheses never
 * win); the region's model is accepted when inliers / total > 0.9, i.e.
 * 10 * inliers > 9 * total (Alg. 2 end, Sec. III-D text).  Regions without a
 * usable hypothesis report hyp_index = -1. */
int or_ransac_regions(const float *P, const unsigned char *valid, const int *regions, int w,
                      int h, int R, int H, float thr, uint64_t seed, uint64_t frame_idx,
                      or_region_plane *out)
{
    long n = (long)w * h;
    if (w <= 0 || h <= 0 || R <= 0 || H <= 0 || !(thr > 0.0f))
        return -1;
    int *u0 = (int *)malloc(4 * (size_t)R * sizeof(int));
    int *cnt = (int *)calloc((size_t)R, sizeof(int));
    if (!u0 || !cnt) {
        free(u0); free(cnt);
        return -2;
    }
    int *v0 = u0 + R, *u1 = u0 + 2 * R, *v1 = u0 + 3 * R;
    for (int r = 0; r < R; ++r) {
        u0[r] = w; v0[r] = h; u1[r] = -1; v1[r] = -1;
    }
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u) {
            long p = (long)v * w + u;
            int r = regions[p];
            if (r < 0 || r >= R || !(valid[p] & 1))
                continue;
            cnt[r]++;
            if (u < u0[r]) u0[r] = u;
            if (u > u1[r]) u1[r] = u;
            if (v < v0[r]) v0[r] = v;
            if (v > v1[r]) v1[r] = v;
        }
    const float thr2 = thr * thr;
    const float scale = 4294967296.0f;   /* 2^32 */
    for (int r = 0; r < R; ++r) {
        or_region_plane *o = &out[r];
        memset(o, 0, sizeof(*o));
        o->total = cnt[r];
        o->hyp_index = -1;
        if (cnt[r] < 3)
            continue;
        unsigned long long best_err = 0;
        int best = -1, best_in = 0;
        float best_pl[4] = {0, 0, 0, 0};
        for (int hh = 0; hh < H; ++hh) {
            long s[3];
            if (!region_sample(seed, frame_idx, r, hh, u0[r], v0[r], u1[r] - u0[r] + 1,
                               v1[r] - v0[r] + 1, w, regions, valid, s))
                continue;
            float q[3][3], pl[4];
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    q[j][k] = P[k * n + s[j]];
            if (!hyp_plane_f32(q[0], q[1], q[2], pl))
                continue;
            unsigned long long err = 0;
            int in = 0;
            for (long p = 0; p < n; ++p) {
                if (regions[p] != r || !(valid[p] & 1))
                    continue;
                float res = fmaf(pl[0], P[p], pl[3]);
                res = fmaf(pl[1], P[n + p], res);
                res = fmaf(pl[2], P[2 * n + p], res);
                float dist = fabsf(res);
                err += (unsigned long long)(dist * scale);
                in += fmaf(res, res, -thr2) < 0.0f;
            }
            if (best < 0 || err < best_err) {
                best = hh;
                best_err = err;
                best_in = in;
                memcpy(best_pl, pl, sizeof(pl));
            }
        }
        if (best < 0)
            continue;
        for (int k = 0; k < 3; ++k)
            o->n[k] = best_pl[k];
        o->d = best_pl[3];
        o->error = best_err;
        o->inliers = best_in;
        o->accepted = 10LL * best_in > 9LL * cnt[r];
        o->hyp_index = best;
    }
    free(u0);
    free(cnt);
    return R;
}

/* The 3 sample pixels of hypothesis h of region r (test access to the
 * sampling rule).  Returns 1 and fills out[3], or 0 if a sample failed. */
int or_region_samples(const int *regions, const unsigned char *valid, int w, int h, int R, int r,
                      int hyp, uint64_t seed, uint64_t frame_idx, long out[3])
{
    int u0 = w, v0 = h, u1 = -1, v1 = -1;
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u) {
            long p = (long)v * w + u;
            if (regions[p] != r || !(valid[p] & 1))
                continue;
            if (u < u0) u0 = u;
            if (u > u1) u1 = u;
            if (v < v0) v0 = v;
            if (v > v1) v1 = v;
        }
    (void)R;
    if (u1 < 0)
        return 0;
    return region_sample(seed, frame_idx, r, hyp, u0, v0, u1 - u0 + 1, v1 - v0 + 1, w, regions,
                         valid, out);
}

/* ------------------------------------------------------------------------ */
/* Canny edges on the normal image and the regions they bound (Sec. III-D:  */
/* edge detection on the normal vector image, then the planar regions).     */
/* ------------------------------------------------------------------------ */

/* 8-bit code of one normal component n in [-1, 1]:
 *   q = clamp(floor(fma(n, 127.5, 128)), 0, 255)  (FP32 fused multiply-add);
 * an invalid pixel is the zero vector, q = 128 in every channel. */
static int canny_code(float n)
{
    float t = fmaf(n, 127.5f, 128.0f);
    int q = (int)floorf(t);
    return q < 0 ? 0 : q > 255 ? 255 : q;
}

/* Direction sector of the gradient (gx, gy), step 4 below:
 *   0: |gy| < tan(22.5 deg) |gx|  <=>  (|gx| + |gy|)^2 < 2 gx^2   (neighbours (u-1, v), (u+1, v))
 *   2: |gx| < tan(22.5 deg) |gy|  <=>  (|gx| + |gy|)^2 < 2 gy^2   (neighbours (u, v-1), (u, v+1))
 *   1: otherwise, gx gy > 0                                    (neighbours (u-1, v-1), (u+1, v+1))
 *   3: otherwise                                               (neighbours (u-1, v+1), (u+1, v-1)) */
int or_canny_sector(int gx, int gy)
{
    long a = labs((long)gx), b = labs((long)gy), s2 = (a + b) * (a + b);
    if (s2 < 2 * a * a)
        return 0;
    if (s2 < 2 * b * b)
        return 2;
    return (long)gx * gy > 0 ? 1 : 3;
}

/* Edge map of the normal image N (FP32 SoA [3][h][w], validity bit 0 of
 * valid):
 *  1. q_c = canny_code(N_c) per channel (128 where invalid); no smoothing of
 *     its own: the depth was smoothed by the anisotropic diffusion, which
 *     the method applies to make the normal image smooth (Sec. III-C);
 *  2. per channel the 3x3 Sobel derivatives gx (along u, to the right) and
 *     gy (along v, downwards), image borders replicated;
 *  3. per pixel the channel with the largest |gx| + |gy| (ties: the lowest
 *     channel); m = |gx| + |gy|;
 *  4. direction sector of (gx, gy): along u when |gy| < tan(22.5 deg) |gx|,
 *     i.e. (|gx| + |gy|)^2 < 2 gx^2 (exact in integers, never an equality
 *     unless gx = gy = 0); along v when (|gx| + |gy|)^2 < 2 gy^2; otherwise
 *     the diagonal through (u+1, v+1) if gx gy > 0, through (u+1, v-1) if not;
 *  5. non-maximum suppression: kept when m > m(behind) and m >= m(ahead)
 *     along the sector (m = 0 outside the image);
 *  6. kept pixels with m > high are strong, with m > low weak; the edges
 *     are the strong pixels and the weak pixels 8-connected to a strong one
 *     through weak pixels (hysteresis).
 * edges: u8 [h][w], 1 = edge; states (may be NULL): u8 [h][w], the state of
 * step 6 before hysteresis (0 none, 1 weak, 2 strong), for tests.  Returns
 * the number of edge pixels, < 0 on error. */
long or_canny(const float *N, const unsigned char *valid, int w, int h, int low, int high,
              unsigned char *edges, unsigned char *states)
{
    if (w <= 0 || h <= 0 || low < 0 || high < low)
        return -1;
    long n = (long)w * h;
    int *q = (int *)malloc(3 * n * sizeof(int));
    int *m = (int *)malloc(n * sizeof(int));
    unsigned char *sec = (unsigned char *)malloc(n);
    unsigned char *st = (unsigned char *)malloc(n);
    long *stack = (long *)malloc(n * sizeof(long));
    if (!q || !m || !sec || !st || !stack) {
        free(q); free(m); free(sec); free(st); free(stack);
        return -2;
    }
    for (int c = 0; c < 3; ++c)
        for (long p = 0; p < n; ++p)
            q[c * n + p] = (valid[p] & 1) ? canny_code(N[c * n + p]) : 128;
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u) {
            int um = u > 0 ? u - 1 : 0, up = u < w - 1 ? u + 1 : w - 1;
            int vm = v > 0 ? v - 1 : 0, vp = v < h - 1 ? v + 1 : h - 1;
            int best = -1, bgx = 0, bgy = 0;
            for (int c = 0; c < 3; ++c) {
                const int *Q = q + c * n;
#define QQ(uu, vv) Q[(long)(vv) * w + (uu)]
                int gx = (QQ(up, vm) + 2 * QQ(up, v) + QQ(up, vp)) -
                         (QQ(um, vm) + 2 * QQ(um, v) + QQ(um, vp));
                int gy = (QQ(um, vp) + 2 * QQ(u, vp) + QQ(up, vp)) -
                         (QQ(um, vm) + 2 * QQ(u, vm) + QQ(up, vm));
#undef QQ
                int mag = abs(gx) + abs(gy);
                if (mag > best) {
                    best = mag;
                    bgx = gx;
                    bgy = gy;
                }
            }
            long p = (long)v * w + u;
            m[p] = best;
            sec[p] = (unsigned char)or_canny_sector(bgx, bgy);
        }
    static const int du[4][2] = {{-1, 1}, {-1, 1}, {0, 0}, {-1, 1}};
    static const int dv[4][2] = {{0, 0}, {-1, 1}, {-1, 1}, {1, -1}};
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u) {
            long p = (long)v * w + u;
            int s = sec[p];
            int nb[2];
            for (int k = 0; k < 2; ++k) {
                int uu = u + du[s][k], vv = v + dv[s][k];
                nb[k] = (uu < 0 || uu >= w || vv < 0 || vv >= h) ? 0 : m[(long)vv * w + uu];
            }
            int keep = m[p] > nb[0] && m[p] >= nb[1];
            st[p] = !keep ? 0 : m[p] > high ? 2 : m[p] > low ? 1 : 0;
        }
    if (states)
        memcpy(states, st, n);
    long top = 0, count = 0;
    for (long p = 0; p < n; ++p) {
        edges[p] = st[p] == 2;
        if (edges[p])
            stack[top++] = p;
    }
    while (top > 0) {
        long p = stack[--top];
        int u = (int)(p % w), v = (int)(p / w);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int uu = u + dx, vv = v + dy;
                if (uu < 0 || uu >= w || vv < 0 || vv >= h)
                    continue;
                long r = (long)vv * w + uu;
                if (st[r] == 1 && !edges[r]) {
                    edges[r] = 1;
                    stack[top++] = r;
                }
            }
    }
    for (long p = 0; p < n; ++p)
        count += edges[p];
    free(q); free(m); free(sec); free(st); free(stack);
    return count;
}

/* Planar regions bounded by the edges: the 4-connected components of the
 * eligible pixels, which are valid, not edges and, when gap = 1, have no
 * edge among their 8 neighbours (this closes the one-pixel breaks that
 * non-maximum suppression leaves where edge lines meet).  Components with
 * fewer than min_pixels pixels get -1; the others are numbered 0, 1, ... in
 * the raster order of their first pixel.  labels: int32 [h][w].  Returns
 * the number of regions. */
int or_segment(const unsigned char *edges, const unsigned char *valid, int w, int h, int gap,
               int min_pixels, int *labels)
{
    if (w <= 0 || h <= 0 || min_pixels < 1 || gap < 0 || gap > 1)
        return -1;
    long n = (long)w * h;
    long *stack = (long *)malloc(n * sizeof(long));
    long *comp = (long *)malloc(n * sizeof(long));
    unsigned char *ok = (unsigned char *)malloc(n);
    if (!stack || !comp || !ok) {
        free(stack); free(comp); free(ok);
        return -2;
    }
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u) {
            long p = (long)v * w + u;
            int e = 0;
            for (int dy = -gap; dy <= gap; ++dy)
                for (int dx = -gap; dx <= gap; ++dx) {
                    int uu = u + dx, vv = v + dy;
                    if (uu >= 0 && uu < w && vv >= 0 && vv < h && edges[(long)vv * w + uu])
                        e = 1;
                }
            ok[p] = (valid[p] & 1) && !e;
        }
    for (long p = 0; p < n; ++p)
        labels[p] = -2;                            /* -2: not visited */
    int R = 0;
    for (long s = 0; s < n; ++s) {
        if (labels[s] != -2)
            continue;
        if (!ok[s]) {
            labels[s] = -1;
            continue;
        }
        long top = 0, k = 0;
        stack[top++] = s;
        labels[s] = -3;                            /* queued */
        while (top > 0) {
            long p = stack[--top];
            comp[k++] = p;
            int u = (int)(p % w), v = (int)(p / w);
            const int nu[4] = {u - 1, u + 1, u, u}, nv[4] = {v, v, v - 1, v + 1};
            for (int j = 0; j < 4; ++j) {
                if (nu[j] < 0 || nu[j] >= w || nv[j] < 0 || nv[j] >= h)
                    continue;
                long r = (long)nv[j] * w + nu[j];
                if (labels[r] == -2 && ok[r]) {
                    labels[r] = -3;
                    stack[top++] = r;
                }
            }
        }
        int lab = k >= min_pixels ? R++ : -1;
        for (long i = 0; i < k; ++i)
            labels[comp[i]] = lab;
    }
    free(stack);
    free(comp);
    free(ok);
    return R;
}
