// TDOM/DSM reference crop on the GPU (Supp. "TDOM/DSM Reference Crop"): the step before
// the pose solver that turns the global maps and a pose prior into a pixel-aligned 2.5D
// reference and its geo-anchors.
//
//   footprint   crop_rays_kernel: one thread-block cluster per image corner; its threads walk the
//               corner ray's samples s_k = s_min + k s_step (metres along the unit ray),
//               read the DSM bilinearly under each, and reduce to the sample whose height is
//               closest to the surface, arg-min |z_ray(s) - h_DSM(x_ray(s), y_ray(s))|
//               (ties: the nearest sample)
//   homography  crop_geometry_kernel: the origin is the footprint's centroid; the
//               homography mapping the normalised crop square's corners (0,0), (1,0), (1,1),
//               (0,1) to the footprint offsets, in closed form (one thread, FP64)
//   warp + lift crop_warp_kernel: one thread per crop pixel: the homography at the pixel
//               centre gives its map coordinates (the warped coordinate grids); the DSM and the
//               TDOM are read bilinearly there (the same warp for every layer), and the pixel is
//               lifted to the geo-anchor (x - ox, y - oy, D)
//
// Geometry is FP64 throughout (it is a handful of values per crop, and one warp per
// pixel); the map is read in place from device memory (an L2/HBM gather of 4 cells per
// layer and pixel), so the whole crop is a few tens of microseconds.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <math.h>

#include "pilot_internal.cuh"

namespace cg = cooperative_groups;

namespace pilot {
namespace {

constexpr int kRayThreads = 256;
constexpr int kRayCluster = 8;      // CTAs per corner ray (a thread-block cluster)

struct MapView {
    const float* dsm;
    const unsigned char* tdom;
    int H, W;
    double x0, y0, gsd;
};

// Bilinear read between cell centres at array coordinates (col, row); false outside
// [0, W-1] x [0, H-1].  The cell is (min(floor(col), W - 2), min(floor(row), H - 2)).
template <typename T>
__device__ __forceinline__ bool read_bilinear(const T* f, int H, int W, int C, int k, double col, double row,
                                              double* out) {
    if (!(col >= 0.0 && col <= W - 1 && row >= 0.0 && row <= H - 1)) return false;
    int c0 = (int)floor(col), r0 = (int)floor(row);
    c0 = min(c0, W - 2);
    r0 = min(r0, H - 2);
    const double ax = col - c0, ay = row - r0;
    const size_t i00 = ((size_t)r0 * W + c0) * C + k;
    const size_t i10 = i00 + (size_t)W * C;
    const double t00 = (double)__ldg(f + i00), t01 = (double)__ldg(f + i00 + C);
    const double t10 = (double)__ldg(f + i10), t11 = (double)__ldg(f + i10 + C);
    *out = (1.0 - ay) * ((1.0 - ax) * t00 + ax * t01) + ay * ((1.0 - ax) * t10 + ax * t11);
    return true;
}

__device__ __forceinline__ void map_coords(const MapView& m, double x, double y, double* col, double* row) {
    *col = (x - m.x0) / m.gsd - 0.5;
    *row = (y - m.y0) / m.gsd - 0.5;
}

// geometry layout: H[9], origin[2], quad[12], sample index per corner (as double, -1: none),
// then 1.0 when the crop is valid (27 values + flag)
constexpr int kGeoH = 0, kGeoOrigin = 9, kGeoQuad = 11, kGeoIdx = 23, kGeoOk = 27;

// Smaller distance first, then the nearer sample.
__device__ __forceinline__ void argmin_merge(double& best, int& arg, double eo, int ko) {
    if (ko >= 0 && (arg < 0 || eo < best || (eo == best && ko < arg))) {
        best = eo;
        arg = ko;
    }
}

// One cluster of kRayCluster CTAs per image corner: CTA r of the cluster takes the samples
// k = r kRayThreads + tid + j kRayCluster kRayThreads (increasing k per thread), reduces to
// its own arg-min, and CTA 0 merges the cluster's results through distributed shared memory.
__global__ void __cluster_dims__(kRayCluster, 1, 1)
crop_rays_kernel(const MapView m, const pilot_crop_params p, double* geometry) {
    __shared__ double s_e[kRayThreads / 32];
    __shared__ int s_k[kRayThreads / 32];
    __shared__ double blk_e;
    __shared__ int blk_k;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int corner = blockIdx.x / kRayCluster;
    const double* T = p.T_cw;
    double Cw[3], d[3];
    for (int i = 0; i < 3; ++i) Cw[i] = -(T[i] * T[3] + T[4 + i] * T[7] + T[8 + i] * T[11]);
    const double u = (corner == 1 || corner == 2) ? (double)p.img_w : 0.0;
    const double v = (corner >= 2) ? (double)p.img_h : 0.0;
    const double dc[3] = {(u - p.cx) / p.fx, (v - p.cy) / p.fy, 1.0};
    for (int i = 0; i < 3; ++i) d[i] = T[i] * dc[0] + T[4 + i] * dc[1] + T[8 + i] * dc[2];
    const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) d[i] /= n;
    double best = INFINITY;
    int arg = -1;
    for (int k = rank * kRayThreads + threadIdx.x; k < p.n_samples; k += kRayCluster * kRayThreads) {
        const double t = p.s_min + k * p.s_step;
        double col, row, h;
        map_coords(m, Cw[0] + t * d[0], Cw[1] + t * d[1], &col, &row);
        if (!read_bilinear(m.dsm, m.H, m.W, 1, 0, col, row, &h)) continue;
        const double e = fabs(Cw[2] + t * d[2] - h);
        if (e < best) {
            best = e;
            arg = k;
        }
    }
    for (int off = 16; off > 0; off >>= 1)
        argmin_merge(best, arg, __shfl_down_sync(0xffffffffu, best, off), __shfl_down_sync(0xffffffffu, arg, off));
    if ((threadIdx.x & 31) == 0) {
        s_e[threadIdx.x >> 5] = best;
        s_k[threadIdx.x >> 5] = arg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kRayThreads / 32; ++w) argmin_merge(best, arg, s_e[w], s_k[w]);
        blk_e = best;
        blk_k = arg;
    }
    cluster.sync();                       // every CTA's result is in its shared memory
    if (rank == 0 && threadIdx.x == 0) {
        for (int r = 1; r < kRayCluster; ++r)
            argmin_merge(best, arg, *cluster.map_shared_rank(&blk_e, r), *cluster.map_shared_rank(&blk_k, r));
        double* q = geometry + kGeoQuad + 3 * corner;
        if (arg < 0) {
            q[0] = q[1] = q[2] = 0.0;
        } else {
            const double t = p.s_min + arg * p.s_step;
            for (int i = 0; i < 3; ++i) q[i] = Cw[i] + t * d[i];
        }
        geometry[kGeoIdx + corner] = (double)arg;
    }
    cluster.sync();                       // keep the shared results alive until they are read
}

// The homography from the unit square's corners (0,0), (1,0), (1,1), (0,1) to the footprint
// offsets p0..p3 in closed form (the square-to-quadrilateral projective map, Heckbert 1989,
// "Fundamentals of Texture Mapping and Image Warping", Sec. 2.2.3), with H[8] = 1; it is the
// unique homography through the four correspondences, the one the 8 x 8 DLT system defines.
__global__ void crop_geometry_kernel(double* geometry) {
    if (threadIdx.x != 0) return;
    double* g = geometry;
    bool ok = true;
    for (int k = 0; k < 4; ++k) ok = ok && g[kGeoIdx + k] >= 0.0;
    double ox = 0.0, oy = 0.0;
    for (int k = 0; k < 4; ++k) {
        ox += g[kGeoQuad + 3 * k];
        oy += g[kGeoQuad + 3 * k + 1];
    }
    ox /= 4.0;
    oy /= 4.0;
    double x[4], y[4];
    for (int k = 0; k < 4; ++k) {
        x[k] = g[kGeoQuad + 3 * k] - ox;
        y[k] = g[kGeoQuad + 3 * k + 1] - oy;
    }
    const double sx = x[0] - x[1] + x[2] - x[3], sy = y[0] - y[1] + y[2] - y[3];
    double a, b, c, d, e, f, gg = 0.0, hh = 0.0;
    if (sx == 0.0 && sy == 0.0) {          // a parallelogram: affine
        a = x[1] - x[0];
        b = x[3] - x[0];
        d = y[1] - y[0];
        e = y[3] - y[0];
    } else {
        const double dx1 = x[1] - x[2], dx2 = x[3] - x[2], dy1 = y[1] - y[2], dy2 = y[3] - y[2];
        const double den = dx1 * dy2 - dx2 * dy1;
        if (den == 0.0) ok = false;
        gg = ok ? (sx * dy2 - dx2 * sy) / den : 0.0;
        hh = ok ? (dx1 * sy - sx * dy1) / den : 0.0;
        a = x[1] - x[0] + gg * x[1];
        b = x[3] - x[0] + hh * x[3];
        d = y[1] - y[0] + gg * y[1];
        e = y[3] - y[0] + hh * y[3];
    }
    c = x[0];
    f = y[0];
    const double Hm[9] = {a, b, c, d, e, f, gg, hh, 1.0};
    for (int i = 0; i < 9; ++i) g[kGeoH + i] = ok ? Hm[i] : 0.0;
    g[kGeoOrigin] = ok ? ox : 0.0;
    g[kGeoOrigin + 1] = ok ? oy : 0.0;
    g[kGeoOk] = ok ? 1.0 : 0.0;
}

__global__ void crop_warp_kernel(const MapView m, int S, const double* __restrict__ geometry, float* points,
                                 unsigned char* valid, float* rgb) {
    const long long NP = (long long)S * S;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NP) return;
    const int u = (int)(j % S), v = (int)(j / S);
    const double* H = geometry + kGeoH;
    bool ok = geometry[kGeoOk] != 0.0;
    double dx = 0.0, dy = 0.0, h = 0.0, col = 0.0, row = 0.0;
    if (ok) {
        const double a = (u + 0.5) / S, b = (v + 0.5) / S;
        const double w = H[6] * a + H[7] * b + H[8];
        dx = (H[0] * a + H[1] * b + H[2]) / w;
        dy = (H[3] * a + H[4] * b + H[5]) / w;
        map_coords(m, geometry[kGeoOrigin] + dx, geometry[kGeoOrigin + 1] + dy, &col, &row);
        ok = w > 0.0 && read_bilinear(m.dsm, m.H, m.W, 1, 0, col, row, &h);
    }
    valid[j] = ok ? 1 : 0;
    points[j] = ok ? (float)dx : 0.0f;
    points[NP + j] = ok ? (float)dy : 0.0f;
    points[2 * NP + j] = ok ? (float)h : 0.0f;
    if (rgb)
        for (int k = 0; k < 3; ++k) {
            double c = 0.0;
            if (ok && m.tdom) read_bilinear(m.tdom, m.H, m.W, 3, k, col, row, &c);
            rgb[3 * j + k] = (float)c;
        }
}

pilot_status crop_fail(pilot_status st, const char* m) {
    record_error(m);
    return st;
}

}  // namespace
}  // namespace pilot

using namespace pilot;

extern "C" pilot_status pilot_crop_reference(const pilot_map* map, const pilot_crop_params* p, float* points,
                                             unsigned char* valid, float* rgb, double* geometry, void* stream) {
    if (!map || !p) return crop_fail(PILOT_EINVAL, "map or params is NULL");
    if (!map->dsm) return crop_fail(PILOT_EINVAL, "the map has no DSM");
    if (map->H < 2 || map->W < 2 || !(map->gsd > 0.0)) return crop_fail(PILOT_EINVAL, "map must be at least 2 x 2 with gsd > 0");
    if (p->S < 1 || p->S > 8192) return crop_fail(PILOT_EINVAL, "crop side S must be in [1, 8192]");
    if (p->n_samples < 1 || p->n_samples > (1 << 22)) return crop_fail(PILOT_EINVAL, "n_samples must be in [1, 4194304]");
    if (!(p->s_step > 0.0) || !(p->fx > 0.0) || !(p->fy > 0.0) || p->img_w < 1 || p->img_h < 1)
        return crop_fail(PILOT_EINVAL, "s_step, fx, fy and the image size must be positive");
    if (!points || !valid || !geometry) return crop_fail(PILOT_EINVAL, "points, valid or geometry is NULL");
    if (((uintptr_t)geometry & 7) != 0 || ((uintptr_t)points & 3) != 0 || (rgb && ((uintptr_t)rgb & 3) != 0))
        return crop_fail(PILOT_EINVAL, "outputs must be naturally aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const MapView m{map->dsm, map->tdom, map->H, map->W, map->x0, map->y0, map->gsd};
    crop_rays_kernel<<<4 * kRayCluster, kRayThreads, 0, s>>>(m, *p, geometry);
    crop_geometry_kernel<<<1, 32, 0, s>>>(geometry);
    const long long NP = (long long)p->S * p->S;
    crop_warp_kernel<<<(unsigned)((NP + 255) / 256), 256, 0, s>>>(m, p->S, geometry, points, valid, rgb);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return crop_fail(PILOT_ECUDA, cudaGetErrorString(e));
    return PILOT_OK;
}
