/*
 * FP64 CPU oracle of the TDOM/DSM reference crop (Supp. "TDOM/DSM Reference Crop").
 * TEST INFRASTRUCTURE ONLY; see crop_oracle.h for the conventions and pins.
 */
#include "crop_oracle.h"

#include <math.h>
#include <string.h>

/* Bilinear read of channel k of an H x W x C map (float or byte) at array coordinates
 * (col, row); 0 when outside [0, W - 1] x [0, H - 1]. */
static int read_bilinear(const float* f, const unsigned char* b, int H, int W, int C, int k, double col,
                         double row, double* out) {
    if (!(col >= 0.0 && col <= W - 1 && row >= 0.0 && row <= H - 1)) return 0;
    int c0 = (int)floor(col), r0 = (int)floor(row);
    if (c0 > W - 2) c0 = W - 2;
    if (r0 > H - 2) r0 = H - 2;
    const double ax = col - c0, ay = row - r0;
    double t[4];
    const long idx[4] = {((long)r0 * W + c0) * C + k, ((long)r0 * W + c0 + 1) * C + k,
                         ((long)(r0 + 1) * W + c0) * C + k, ((long)(r0 + 1) * W + c0 + 1) * C + k};
    for (int i = 0; i < 4; ++i) t[i] = f ? (double)f[idx[i]] : (double)b[idx[i]];
    *out = (1.0 - ay) * ((1.0 - ax) * t[0] + ax * t[1]) + ay * ((1.0 - ax) * t[2] + ax * t[3]);
    return 1;
}

static void map_coords(const orc_map* m, double x, double y, double* col, double* row) {
    *col = (x - m->x0) / m->gsd - 0.5;
    *row = (y - m->y0) / m->gsd - 0.5;
}

int orc_dsm_height(const orc_map* m, double x, double y, double* h) {
    double col, row;
    map_coords(m, x, y, &col, &row);
    *h = 0.0;
    return read_bilinear(m->dsm, NULL, m->H, m->W, 1, 0, col, row, h);
}

void orc_footprint(const orc_map* m, const orc_params* p, double quad[12], int idx[4]) {
    const double* T = p->T_cw;
    /* camera centre C = -R^T t */
    double Cw[3];
    for (int i = 0; i < 3; ++i) Cw[i] = -(T[i] * T[3] + T[4 + i] * T[7] + T[8 + i] * T[11]);
    const double cu[4] = {0.0, (double)p->img_w, (double)p->img_w, 0.0};
    const double cv[4] = {0.0, 0.0, (double)p->img_h, (double)p->img_h};
    for (int k = 0; k < 4; ++k) {
        /* direction R^T K^-1 [u, v, 1], unit length */
        const double dc[3] = {(cu[k] - p->cx) / p->fx, (cv[k] - p->cy) / p->fy, 1.0};
        double d[3];
        for (int i = 0; i < 3; ++i) d[i] = T[i] * dc[0] + T[4 + i] * dc[1] + T[8 + i] * dc[2];
        const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) d[i] /= n;
        double best = INFINITY;
        int arg = -1;
        for (int s = 0; s < p->n_samples; ++s) {
            const double t = p->s_min + s * p->s_step;
            const double x = Cw[0] + t * d[0], y = Cw[1] + t * d[1], z = Cw[2] + t * d[2];
            double h;
            if (!orc_dsm_height(m, x, y, &h)) continue;
            const double e = fabs(z - h);
            if (e < best) {
                best = e;
                arg = s;
            }
        }
        idx[k] = arg;
        if (arg < 0) {
            quad[3 * k] = quad[3 * k + 1] = quad[3 * k + 2] = 0.0;
        } else {
            const double t = p->s_min + arg * p->s_step;
            for (int i = 0; i < 3; ++i) quad[3 * k + i] = Cw[i] + t * d[i];
        }
    }
}

int orc_homography(const double src[8], const double dst[8], double H[9]) {
    /* rows: [u v 1 0 0 0 -u x -v x | x] and [0 0 0 u v 1 -u y -v y | y] */
    double A[8][9];
    for (int i = 0; i < 4; ++i) {
        const double u = src[2 * i], v = src[2 * i + 1], x = dst[2 * i], y = dst[2 * i + 1];
        const double r0[9] = {u, v, 1.0, 0.0, 0.0, 0.0, -u * x, -v * x, x};
        const double r1[9] = {0.0, 0.0, 0.0, u, v, 1.0, -u * y, -v * y, y};
        memcpy(A[2 * i], r0, sizeof r0);
        memcpy(A[2 * i + 1], r1, sizeof r1);
    }
    for (int c = 0; c < 8; ++c) {
        int piv = c;
        for (int r = c + 1; r < 8; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return 0;
        if (piv != c)
            for (int j = 0; j < 9; ++j) {
                const double tmp = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = tmp;
            }
        for (int r = c + 1; r < 8; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int j = c; j < 9; ++j) A[r][j] -= f * A[c][j];
        }
    }
    double h[8];
    for (int c = 7; c >= 0; --c) {
        double s = A[c][8];
        for (int j = c + 1; j < 8; ++j) s -= A[c][j] * h[j];
        h[c] = s / A[c][c];
    }
    for (int i = 0; i < 8; ++i) H[i] = h[i];
    H[8] = 1.0;
    return 1;
}

void orc_warp(const orc_map* m, const double H[9], int S, double ox, double oy, float* points,
              unsigned char* valid, float* rgb) {
    const long NP = (long)S * S;
    for (int v = 0; v < S; ++v)
        for (int u = 0; u < S; ++u) {
            const long j = (long)v * S + u;
            const double a = (u + 0.5) / S, b = (v + 0.5) / S;
            const double w = H[6] * a + H[7] * b + H[8];
            const double dx = (H[0] * a + H[1] * b + H[2]) / w;
            const double dy = (H[3] * a + H[4] * b + H[5]) / w;
            double col, row, h = 0.0;
            map_coords(m, ox + dx, oy + dy, &col, &row);
            const int ok = w > 0.0 && read_bilinear(m->dsm, NULL, m->H, m->W, 1, 0, col, row, &h);
            valid[j] = (unsigned char)ok;
            points[j] = ok ? (float)dx : 0.0f;
            points[NP + j] = ok ? (float)dy : 0.0f;
            points[2 * NP + j] = ok ? (float)h : 0.0f;
            if (rgb) {
                for (int k = 0; k < 3; ++k) {
                    double c = 0.0;
                    if (ok && m->tdom) read_bilinear(NULL, m->tdom, m->H, m->W, 3, k, col, row, &c);
                    rgb[3 * j + k] = (float)c;
                }
            }
        }
}

int orc_crop(const orc_map* m, const orc_params* p, double geometry[27], float* points,
             unsigned char* valid, float* rgb) {
    double quad[12];
    int idx[4];
    orc_footprint(m, p, quad, idx);
    memset(geometry, 0, 27 * sizeof(double));
    for (int k = 0; k < 12; ++k) geometry[11 + k] = quad[k];
    for (int k = 0; k < 4; ++k) geometry[23 + k] = idx[k];
    const long NP = (long)p->S * p->S;
    int ok = idx[0] >= 0 && idx[1] >= 0 && idx[2] >= 0 && idx[3] >= 0;
    double ox = 0.0, oy = 0.0, H[9] = {0};
    if (ok) {
        for (int k = 0; k < 4; ++k) {
            ox += quad[3 * k];
            oy += quad[3 * k + 1];
        }
        ox /= 4.0;
        oy /= 4.0;
        const double src[8] = {0.0, 0.0, 1.0, 0.0, 1.0, 1.0, 0.0, 1.0};
        double dst[8];
        for (int k = 0; k < 4; ++k) {
            dst[2 * k] = quad[3 * k] - ox;
            dst[2 * k + 1] = quad[3 * k + 1] - oy;
        }
        ok = orc_homography(src, dst, H);
    }
    if (!ok) {
        memset(points, 0, 3 * NP * sizeof(float));
        memset(valid, 0, NP);
        if (rgb) memset(rgb, 0, 3 * NP * sizeof(float));
        return 0;
    }
    for (int i = 0; i < 9; ++i) geometry[i] = H[i];
    geometry[9] = ox;
    geometry[10] = oy;
    orc_warp(m, H, p->S, ox, oy, points, valid, rgb);
    return 1;
}
