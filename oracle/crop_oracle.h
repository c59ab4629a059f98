/*
 * FP64 CPU oracle of the TDOM/DSM reference crop (Supp. "TDOM/DSM Reference Crop"): the
 * step that turns the global maps and a pose prior into the pixel-aligned 2.5D reference
 * and its geo-anchors.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain loops in double precision, in the order the paper
 * states the three steps; only the test suite and the benchmark's CPU-baseline leg may
 * load it.  It shares no code with the CUDA library.
 *
 *   map footprint   the four corner rays of the image, each at the ray sample whose height
 *                   is closest to the DSM surface (the arg-min of |z_ray(s) - h_DSM| over
 *                   the samples)
 *   warping         the homography from the crop square to that footprint quadrilateral,
 *                   applied to the TDOM, the DSM and the map-coordinate grids alike
 *   geo-anchors     P(u, v) = (x_m(u, v), y_m(u, v), D_r(u, v)) for every valid crop pixel
 *
 * Conventions (readings, listed in the design notes): the map's cell (r, c) is centred at
 * (x0 + (c + 1/2) gsd, y0 + (r + 1/2) gsd) and the DSM is read bilinearly between cell
 * centres (cell c0 = min(floor(col), W - 2)); the corner rays go through the image corners
 * (0, 0), (W, 0), (W, H), (0, H) (pixel i covers [i, i + 1)), which map to the crop corners
 * (0, 0), (S, 0), (S, S), (0, S); ray samples are s_k = s_min + k s_step metres along the
 * unit ray, k = 0 .. n_samples - 1, samples off the DSM excluded; the homography maps the
 * normalised crop coordinates (u / S, v / S) to metric offsets from the origin, the centroid
 * of the four footprint points; crop pixel (u, v) is read at its centre (u + 1/2, v + 1/2).
 *
 * Pinned by: a flat DSM (footprint = the closed-form ray-plane intersections within one
 * sample), the homography's exact corner mapping, exactness of bilinear warping on affine
 * maps, and every anchor lying on the bilinear DSM surface.
 */
#ifndef CROP_ORACLE_H
#define CROP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    const float* dsm;             /* H x W heights (metres), row-major */
    const unsigned char* tdom;    /* H x W x 3 RGB, or NULL */
    int H, W;
    double x0, y0, gsd;
} orc_map;

typedef struct {
    double T_cw[12];              /* pose prior [R | t], world -> camera, row-major */
    double fx, fy, cx, cy;        /* image intrinsics, pixel-corner convention */
    int img_w, img_h;
    double s_min, s_step;
    int n_samples;
    int S;                        /* crop side in pixels */
} orc_params;

/* Bilinear DSM height at metric (x, y); 0 when (x, y) is outside the cell-centre grid. */
int orc_dsm_height(const orc_map* m, double x, double y, double* h);

/* Footprint: quad[3k .. 3k + 2] = the sample of corner ray k closest to the DSM, idx[k] its
 * sample index (-1 when no sample of the ray lies over the DSM). */
void orc_footprint(const orc_map* m, const orc_params* p, double quad[12], int idx[4]);

/* Homography with src[2i], src[2i + 1] -> dst[2i], dst[2i + 1] for the four i (DLT with
 * H[8] = 1, Gaussian elimination with partial pivoting).  0 if singular. */
int orc_homography(const double src[8], const double dst[8], double H[9]);

/* Warp of one crop: for pixel (u, v) (index v S + u), points[0..2][.] = (x - ox, y - oy, D),
 * valid = inside the cell-centre grid, rgb[3 (v S + u) + k] = bilinear TDOM channel k (if both
 * rgb and the map's TDOM are given).  Invalid pixels get zeros. */
void orc_warp(const orc_map* m, const double H[9], int S, double ox, double oy, float* points,
              unsigned char* valid, float* rgb);

/* The three steps: footprint, homography (origin = footprint centroid), warp.  geometry
 * receives H[9], origin[2], quad[12] and the four sample indices (as doubles), 27 values.
 * Returns 0 when a corner ray misses the DSM (outputs zeroed), else 1. */
int orc_crop(const orc_map* m, const orc_params* p, double geometry[27], float* points,
             unsigned char* valid, float* rgb);

#ifdef __cplusplus
}
#endif

#endif
