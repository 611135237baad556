/*
 * czgen.c -- seeded synthetic fields that stand in for the paper's
 * cloud-cavitation snapshots (Sec. 3.1: Cubism-MPCF HDF5 data of a bubble
 * cloud, not available here).  These generators hold none of the codec's
 * arithmetic; the tests and the benchmark feed the same bytes to the GPU
 * library and to the CPU oracle.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014), written from its
 * published definition; uniform doubles are the top 53 bits times 2^-53;
 * Gaussian noise is Box-Muller on two counter-indexed draws so every point is
 * independent of evaluation order.  Values are formed in double and rounded
 * once to the output type.  Work is split over z-planes (OpenMP); every point
 * is a pure function of its coordinates and the seed.
 *
 * Recipes (cell centres X = i + 1/2):
 *   CZGEN_GAUSS  1 + sum of 8 Gaussian bubbles A exp(-|X-c|^2 / (2 s^2)),
 *                A ~ U[10,100], s ~ U[4,16], c ~ U[0,n) per axis, plus noise
 *                N(0, sigma = 1e-4).
 *   CZGEN_ALPHA  gas fraction of nb bubbles, r ~ U[4,30], c ~ U[0,n):
 *                alpha_b = (1 - tanh(|X-c| - r)) / 2 (interface about two
 *                cells wide), alpha = max_b alpha_b, evaluated where
 *                |X-c| < r + 20 (elsewhere alpha_b < 5e-18 and is taken as 0).
 *   CZGEN_RHO    alpha * 1 + (1 - alpha) * 1000.
 *   CZGEN_P      1e5 + 1e4 * (1/8) sum_{m<8} sin(2 pi k_m.X/n + phi_m)
 *                - 9e4 * alpha, k_m in {-4..4}^3 \ {0}, phi ~ U[0, 2 pi).
 * Draw order: bubbles (c_x, c_y, c_z, r) for ALPHA/RHO/P, then the 8 modes
 * (k_x, k_y, k_z redrawn while all zero, then phi); for GAUSS the 8 bubbles
 * (A, s, c_x, c_y, c_z); then one draw seeds the noise counter.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { CZGEN_GAUSS = 0, CZGEN_ALPHA = 1, CZGEN_RHO = 2, CZGEN_P = 3 };

#define GOLDEN 0x9e3779b97f4a7c15ULL

static uint64_t mix64(uint64_t z)
{
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static uint64_t next64(uint64_t *s)
{
  *s += GOLDEN;
  return mix64(*s);
}

static double unif(uint64_t *s) { return (double)(next64(s) >> 11) * 0x1.0p-53; }

typedef struct {
  double cx, cy, cz, r;
} bubble;

typedef struct {
  double a, s, cx, cy, cz;
} gauss;

typedef struct {
  int kx, ky, kz;
  double phi;
} mode;

static const double TWO_PI = 6.283185307179586476925286766559;

static void store(void *out, int dtype, size_t i, double v)
{
  if (dtype == 1)
    ((double *)out)[i] = v;
  else
    ((float *)out)[i] = (float)v;
}

/* gas fraction of plane z (alpha[y*nx + x]) */
static void alpha_plane(const bubble *bub, int nb, int nx, int ny, int z, double *alpha)
{
  memset(alpha, 0, sizeof(double) * (size_t)nx * ny);
  double Z = z + 0.5;
  for (int b = 0; b < nb; ++b) {
    double R = bub[b].r + 20.0;
    double dz = Z - bub[b].cz;
    if (fabs(dz) >= R) continue;
    int y0 = (int)floor(bub[b].cy - R), y1 = (int)ceil(bub[b].cy + R);
    int x0 = (int)floor(bub[b].cx - R), x1 = (int)ceil(bub[b].cx + R);
    if (y0 < 0) y0 = 0;
    if (x0 < 0) x0 = 0;
    if (y1 > ny - 1) y1 = ny - 1;
    if (x1 > nx - 1) x1 = nx - 1;
    for (int y = y0; y <= y1; ++y) {
      double dy = y + 0.5 - bub[b].cy;
      for (int x = x0; x <= x1; ++x) {
        double dx = x + 0.5 - bub[b].cx;
        double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d >= R) continue;
        double a = 0.5 * (1.0 - tanh(d - bub[b].r));
        double *dst = &alpha[(size_t)y * nx + x];
        if (a > *dst) *dst = a;
      }
    }
  }
}

int czgen_field(int recipe, int dtype, int nx, int ny, int nz, uint64_t seed,
                int nbubbles, void *out)
{
  if (nx <= 0 || ny <= 0 || nz <= 0 || (dtype != 0 && dtype != 1)) return -1;
  if (recipe < CZGEN_GAUSS || recipe > CZGEN_P) return -1;
  uint64_t st = seed;
  const size_t plane = (size_t)nx * ny;

  if (recipe == CZGEN_GAUSS) {
    gauss g[8];
    for (int b = 0; b < 8; ++b) {
      g[b].a = 10.0 + 90.0 * unif(&st);
      g[b].s = 4.0 + 12.0 * unif(&st);
      g[b].cx = nx * unif(&st);
      g[b].cy = ny * unif(&st);
      g[b].cz = nz * unif(&st);
    }
    uint64_t noise = next64(&st);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          double X = x + 0.5, Y = y + 0.5, Zc = z + 0.5;
          double v = 1.0;
          for (int b = 0; b < 8; ++b) {
            double dx = X - g[b].cx, dy = Y - g[b].cy, dz = Zc - g[b].cz;
            v += g[b].a * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * g[b].s * g[b].s));
          }
          size_t i = (size_t)z * plane + (size_t)y * nx + x;
          double u1 = (double)((mix64(noise + (2 * (uint64_t)i + 1) * GOLDEN) >> 11) + 1) * 0x1.0p-53;
          double u2 = (double)(mix64(noise + (2 * (uint64_t)i + 2) * GOLDEN) >> 11) * 0x1.0p-53;
          v += 1e-4 * sqrt(-2.0 * log(u1)) * cos(TWO_PI * u2);
          store(out, dtype, i, v);
        }
    return 0;
  }

  if (nbubbles < 0) return -1;
  bubble *bub = (bubble *)malloc(sizeof(bubble) * (size_t)(nbubbles > 0 ? nbubbles : 1));
  if (!bub) return -1;
  for (int b = 0; b < nbubbles; ++b) {
    bub[b].cx = nx * unif(&st);
    bub[b].cy = ny * unif(&st);
    bub[b].cz = nz * unif(&st);
    bub[b].r = 4.0 + 26.0 * unif(&st);
  }
  mode md[8];
  for (int m = 0; m < 8; ++m) {
    do {
      md[m].kx = (int)floor(9.0 * unif(&st)) - 4;
      md[m].ky = (int)floor(9.0 * unif(&st)) - 4;
      md[m].kz = (int)floor(9.0 * unif(&st)) - 4;
    } while (md[m].kx == 0 && md[m].ky == 0 && md[m].kz == 0);
    md[m].phi = TWO_PI * unif(&st);
  }

  /* per-axis phase factors for the sine modes: e^{i 2 pi k (i+1/2) / n} */
  double *ex = NULL, *ey = NULL, *ez = NULL;
  if (recipe == CZGEN_P) {
    ex = (double *)malloc(sizeof(double) * 2 * 8 * (size_t)nx);
    ey = (double *)malloc(sizeof(double) * 2 * 8 * (size_t)ny);
    ez = (double *)malloc(sizeof(double) * 2 * 8 * (size_t)nz);
    if (!ex || !ey || !ez) {
      free(ex); free(ey); free(ez); free(bub);
      return -1;
    }
    for (int m = 0; m < 8; ++m) {
      for (int i = 0; i < nx; ++i) {
        double a = TWO_PI * md[m].kx * (i + 0.5) / nx;
        ex[2 * (m * (size_t)nx + i)] = cos(a);
        ex[2 * (m * (size_t)nx + i) + 1] = sin(a);
      }
      for (int i = 0; i < ny; ++i) {
        double a = TWO_PI * md[m].ky * (i + 0.5) / ny;
        ey[2 * (m * (size_t)ny + i)] = cos(a);
        ey[2 * (m * (size_t)ny + i) + 1] = sin(a);
      }
      for (int i = 0; i < nz; ++i) {
        double a = TWO_PI * md[m].kz * (i + 0.5) / nz + md[m].phi;
        ez[2 * (m * (size_t)nz + i)] = cos(a);
        ez[2 * (m * (size_t)nz + i) + 1] = sin(a);
      }
    }
  }

  int fail = 0;
#pragma omp parallel
  {
    double *alpha = (double *)malloc(sizeof(double) * plane);
    if (!alpha) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(static)
    for (int z = 0; z < nz; ++z) {
      if (!alpha) continue;
      alpha_plane(bub, nbubbles, nx, ny, z, alpha);
      for (int y = 0; y < ny; ++y) {
        double qr[8], qi[8];
        if (recipe == CZGEN_P)
          for (int m = 0; m < 8; ++m) {
            const double *a = &ez[2 * (m * (size_t)nz + z)];
            const double *b = &ey[2 * (m * (size_t)ny + y)];
            qr[m] = a[0] * b[0] - a[1] * b[1];
            qi[m] = a[0] * b[1] + a[1] * b[0];
          }
        for (int x = 0; x < nx; ++x) {
          size_t i = (size_t)z * plane + (size_t)y * nx + x;
          double al = alpha[(size_t)y * nx + x], v;
          if (recipe == CZGEN_ALPHA) {
            v = al;
          } else if (recipe == CZGEN_RHO) {
            v = al * 1.0 + (1.0 - al) * 1000.0;
          } else {
            double s = 0.0;
            for (int m = 0; m < 8; ++m) {
              const double *c = &ex[2 * (m * (size_t)nx + x)];
              s += qr[m] * c[1] + qi[m] * c[0]; /* Im(q * e_x) */
            }
            v = 1e5 + 1e4 * (0.125 * s) - 9e4 * al;
          }
          store(out, dtype, i, v);
        }
      }
    }
    free(alpha);
  }
  free(ex);
  free(ey);
  free(ez);
  free(bub);
  return fail ? -1 : 0;
}
