/*
 * FP64 reference projector of the oracle (test infrastructure: only tests, the smoke check
 * and the bench's CPU-baseline leg use it; the CUDA library never links or calls it).
 *
 * The projection operator P of the PET problem (Sec. 1.2, Eq. EQU:PROB:OPT) is not specified
 * by the paper beyond its geometric, attenuation and normalisation factors; this file computes
 * its geometric part L as the exact line integral of the piecewise-constant image along each
 * line of response:  (L x)_j = sum_k len(LOR_j  intersect voxel_k) * x_k,  lengths in units of
 * the transaxial voxel size.  Per-bin multipliers are applied by the Python layer.
 *
 * Two independent evaluations of the same definition are provided:
 *   - og_trace: Siddon's parametric method -- all crossings of the LOR with the x, y and z
 *     grid planes are collected, sorted, and each interval between consecutive crossings is
 *     attributed to the voxel containing its mid-point;
 *   - og_clip_len: the length of the LOR inside ONE voxel box by slab clipping.
 * A line lying exactly in a grid plane (a direction component equal to zero) belongs to the
 * voxel whose lower face contains it (half-open voxels [lo, hi)).
 *
 * Geometry conventions (shared with the documented C ABI, implemented here independently):
 * image x[iy][ix][iz]; voxel lower corner X_i = -nx*vx/2 + i*vx (same for y, z);
 * sinogram y[view][radial][plane]; phi_v = v*pi/V with cos/sin values below 1e-12 set to 0;
 * s_r = (r - (R-1)/2)*d_radial; plane q of segment g: z_mid = zmid0[g] + q*dzmid[g];
 * LOR point P(t) = (s cos - t sin, s sin + t cos, z_mid + t*dz/(2h)), t in [-h, h],
 * h = sqrt(radius^2 - s^2).
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nx, ny, nz;
  double vx, vy, vz;
  int n_radial;
  double d_radial;
  int n_views;
  double radius;
  int n_seg;
  const int* seg_n;
  const double* seg_zmid0;
  const double* seg_dzmid;
  const double* seg_dz;
  int n_subsets;
} og_geom;

int og_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int og_n_planes(const og_geom* g) {
  int p = 0;
  for (int k = 0; k < g->n_seg; ++k) p += g->seg_n[k];
  return p;
}

static void og_plane(const og_geom* g, int p, double* zm, double* dz) {
  for (int k = 0; k < g->n_seg; ++k) {
    if (p < g->seg_n[k]) {
      *zm = g->seg_zmid0[k] + p * g->seg_dzmid[k];
      *dz = g->seg_dz[k];
      return;
    }
    p -= g->seg_n[k];
  }
  *zm = 0.0;
  *dz = 0.0;
}

static void og_lor(const og_geom* g, int v, int r, int p, double o[3], double d[3], double* h) {
  double phi = 3.14159265358979323846 * (double)v / (double)g->n_views;
  double c = cos(phi), sn = sin(phi);
  if (fabs(c) < 1e-12) c = 0.0;
  if (fabs(sn) < 1e-12) sn = 0.0;
  double s = (r - 0.5 * (g->n_radial - 1)) * g->d_radial;
  double zm, dz;
  og_plane(g, p, &zm, &dz);
  *h = sqrt(g->radius * g->radius - s * s);
  o[0] = s * c;
  o[1] = s * sn;
  o[2] = zm;
  d[0] = -sn;
  d[1] = c;
  d[2] = dz / (2.0 * (*h));
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* Siddon: voxels crossed by the LOR and their lengths. idx/len/tb hold nx+ny+nz+2 entries. */
static int og_trace(const og_geom* g, const double o[3], const double d[3], double h, long* idx,
                    double* len, double* tb) {
  const int n[3] = {g->nx, g->ny, g->nz};
  const double v[3] = {g->vx, g->vy, g->vz};
  double lo[3], hi[3];
  double t0 = -h, t1 = h;
  for (int a = 0; a < 3; ++a) {
    lo[a] = -n[a] * v[a] / 2.0;
    hi[a] = n[a] * v[a] / 2.0;
    if (d[a] == 0.0) {
      if (o[a] < lo[a] || o[a] >= hi[a]) return 0;
    } else {
      double ta = (lo[a] - o[a]) / d[a], tc = (hi[a] - o[a]) / d[a];
      t0 = fmax(t0, fmin(ta, tc));
      t1 = fmin(t1, fmax(ta, tc));
    }
  }
  if (!(t0 < t1)) return 0;
  int m = 0;
  tb[m++] = t0;
  tb[m++] = t1;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0) continue;
    for (int k = 1; k < n[a]; ++k) {
      double t = (lo[a] + k * v[a] - o[a]) / d[a];
      if (t > t0 && t < t1) tb[m++] = t;
    }
  }
  qsort(tb, (size_t)m, sizeof(double), cmp_double);
  const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  int cnt = 0;
  for (int k = 0; k + 1 < m; ++k) {
    if (!(tb[k + 1] > tb[k])) continue;
    double tm = 0.5 * (tb[k] + tb[k + 1]);
    int i[3];
    for (int a = 0; a < 3; ++a) {
      double c = (d[a] == 0.0) ? o[a] : o[a] + tm * d[a];
      int ii = (int)floor((c - lo[a]) / v[a]);
      if (ii < 0) ii = 0;
      if (ii >= n[a]) ii = n[a] - 1;
      i[a] = ii;
    }
    idx[cnt] = ((long)i[1] * g->nx + i[0]) * g->nz + i[2];
    len[cnt] = (tb[k + 1] - tb[k]) * dn / g->vx;
    ++cnt;
  }
  return cnt;
}

/* Length of the LOR inside voxel (ix, iy, iz) by slab clipping (voxel-size units). */
static double og_clip_len(const og_geom* g, const double o[3], const double d[3], double h, int ix,
                          int iy, int iz) {
  const int n[3] = {g->nx, g->ny, g->nz};
  const double v[3] = {g->vx, g->vy, g->vz};
  const int i[3] = {ix, iy, iz};
  double t0 = -h, t1 = h;
  for (int a = 0; a < 3; ++a) {
    double lo = -n[a] * v[a] / 2.0 + i[a] * v[a];
    double hi = -n[a] * v[a] / 2.0 + (i[a] + 1) * v[a];
    if (d[a] == 0.0) {
      if (o[a] < lo || o[a] >= hi) return 0.0;
    } else {
      double ta = (lo - o[a]) / d[a], tc = (hi - o[a]) / d[a];
      t0 = fmax(t0, fmin(ta, tc));
      t1 = fmin(t1, fmax(ta, tc));
    }
  }
  if (!(t1 > t0)) return 0.0;
  return (t1 - t0) * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / g->vx;
}

static int og_in_subset(const og_geom* g, int v, int subset) {
  return subset < 0 || (v % g->n_subsets) == subset;
}

/* y[j] = (L x)_j for every bin j of the subset (subset < 0: all bins); other bins untouched. */
void og_project(const og_geom* g, const double* x, double* y, int subset) {
  const int R = g->n_radial, P = og_n_planes(g), V = g->n_views;
  const int nbuf = g->nx + g->ny + g->nz + 4;
  const long nb = (long)V * R * P;
#pragma omp parallel
  {
    long* idx = (long*)malloc(sizeof(long) * nbuf);
    double* len = (double*)malloc(sizeof(double) * nbuf);
    double* tb = (double*)malloc(sizeof(double) * nbuf);
#pragma omp for schedule(dynamic, 64)
    for (long j = 0; j < nb; ++j) {
      int v = (int)(j / ((long)R * P));
      if (!og_in_subset(g, v, subset)) continue;
      int r = (int)((j / P) % R), p = (int)(j % P);
      double o[3], d[3], h;
      og_lor(g, v, r, p, o, d, &h);
      int c = og_trace(g, o, d, h, idx, len, tb);
      double acc = 0.0;
      for (int k = 0; k < c; ++k) acc += len[k] * x[idx[k]];
      y[j] = acc;
    }
    free(idx);
    free(len);
    free(tb);
  }
}

/* x = L_subset^T y (x is overwritten).  Serial scatter along the same traversal. */
void og_backproject(const og_geom* g, const double* y, double* x, int subset) {
  const int R = g->n_radial, P = og_n_planes(g), V = g->n_views;
  const int nbuf = g->nx + g->ny + g->nz + 4;
  memset(x, 0, sizeof(double) * (size_t)g->nx * g->ny * g->nz);
  long* idx = (long*)malloc(sizeof(long) * nbuf);
  double* len = (double*)malloc(sizeof(double) * nbuf);
  double* tb = (double*)malloc(sizeof(double) * nbuf);
  for (int v = 0; v < V; ++v) {
    if (!og_in_subset(g, v, subset)) continue;
    for (int r = 0; r < R; ++r)
      for (int p = 0; p < P; ++p) {
        long j = ((long)v * R + r) * P + p;
        if (y[j] == 0.0) continue;
        double o[3], d[3], h;
        og_lor(g, v, r, p, o, d, &h);
        int c = og_trace(g, o, d, h, idx, len, tb);
        for (int k = 0; k < c; ++k) x[idx[k]] += len[k] * y[j];
      }
  }
  free(idx);
  free(len);
  free(tb);
}

/* out[k] = (L x)_{bins[k]} for a list of full-sinogram bin indices. */
void og_project_bins(const og_geom* g, const double* x, long n, const long* bins, double* out) {
  const int R = g->n_radial, P = og_n_planes(g);
  const int nbuf = g->nx + g->ny + g->nz + 4;
#pragma omp parallel
  {
    long* idx = (long*)malloc(sizeof(long) * nbuf);
    double* len = (double*)malloc(sizeof(double) * nbuf);
    double* tb = (double*)malloc(sizeof(double) * nbuf);
#pragma omp for schedule(dynamic, 16)
    for (long k = 0; k < n; ++k) {
      long j = bins[k];
      int v = (int)(j / ((long)R * P)), r = (int)((j / P) % R), p = (int)(j % P);
      double o[3], d[3], h;
      og_lor(g, v, r, p, o, d, &h);
      int c = og_trace(g, o, d, h, idx, len, tb);
      double acc = 0.0;
      for (int q = 0; q < c; ++q) acc += len[q] * x[idx[q]];
      out[k] = acc;
    }
    free(idx);
    free(len);
    free(tb);
  }
}

/* out[k] = (L_subset^T y)_{voxels[k]} by the definition: sum over every LOR of the subset of
 * (slab-clipped length inside that voxel) * y. */
void og_backproject_voxels(const og_geom* g, const double* y, int subset, long n, const long* voxels,
                           double* out) {
  const int R = g->n_radial, P = og_n_planes(g), V = g->n_views;
#pragma omp parallel for schedule(dynamic, 1)
  for (long k = 0; k < n; ++k) {
    long vox = voxels[k];
    int iz = (int)(vox % g->nz);
    int ix = (int)((vox / g->nz) % g->nx);
    int iy = (int)(vox / ((long)g->nz * g->nx));
    double acc = 0.0;
    for (int v = 0; v < V; ++v) {
      if (!og_in_subset(g, v, subset)) continue;
      for (int r = 0; r < R; ++r)
        for (int p = 0; p < P; ++p) {
          long j = ((long)v * R + r) * P + p;
          double o[3], d[3], h;
          og_lor(g, v, r, p, o, d, &h);
          double l = og_clip_len(g, o, d, h, ix, iy, iz);
          if (l != 0.0) acc += l * y[j];
        }
    }
    out[k] = acc;
  }
}

/* Dense system matrix by slab clipping, rows = bins (all), cols = voxels.  Tiny cases only. */
void og_dense_clip(const og_geom* g, double* A) {
  const int R = g->n_radial, P = og_n_planes(g), V = g->n_views;
  const long N = (long)g->nx * g->ny * g->nz;
  for (int v = 0; v < V; ++v)
    for (int r = 0; r < R; ++r)
      for (int p = 0; p < P; ++p) {
        long j = ((long)v * R + r) * P + p;
        double o[3], d[3], h;
        og_lor(g, v, r, p, o, d, &h);
        for (int iy = 0; iy < g->ny; ++iy)
          for (int ix = 0; ix < g->nx; ++ix)
            for (int iz = 0; iz < g->nz; ++iz)
              A[j * N + ((long)iy * g->nx + ix) * g->nz + iz] = og_clip_len(g, o, d, h, ix, iy, iz);
      }
}

/* out[k * n_subsets + i] = (L_i^T w)_{voxels[k]} for every subset i, by the definition (slab-
 * clipped length of every LOR inside the voxel), in one pass over the bins. */
void og_subset_sums_at_voxels(const og_geom* g, const double* w, long n, const long* voxels, double* out) {
  const int R = g->n_radial, P = og_n_planes(g), V = g->n_views, m = g->n_subsets;
#pragma omp parallel for schedule(dynamic, 1)
  for (long k = 0; k < n; ++k) {
    long vox = voxels[k];
    int iz = (int)(vox % g->nz);
    int ix = (int)((vox / g->nz) % g->nx);
    int iy = (int)(vox / ((long)g->nz * g->nx));
    for (int i = 0; i < m; ++i) out[k * m + i] = 0.0;
    for (int v = 0; v < V; ++v)
      for (int r = 0; r < R; ++r)
        for (int p = 0; p < P; ++p) {
          long j = ((long)v * R + r) * P + p;
          double o[3], d[3], h;
          og_lor(g, v, r, p, o, d, &h);
          double l = og_clip_len(g, o, d, h, ix, iy, iz);
          if (l != 0.0) out[k * m + (v % m)] += l * w[j];
        }
  }
}
