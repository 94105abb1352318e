/*
 * ibm_oracle.c -- plain, slow, FP64 CPU oracle of the sharp-interface IBM
 * fractional step (Vagnoli, Scarpolini, Verzicco, Viola, arXiv 2606.09799).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * Every function below follows one passage of the paper, cited in its
 * comment.  Loops are written in the plainest order; there is no blocking,
 * fusion or reordering beyond what the cited equation or algorithm states.
 * The discrete Fourier transform of the Poisson solve is done in Python
 * (numpy.fft) by oracle.py; this file holds everything else.
 *
 * Conventions (shared with the CUDA path only through the paper's text and
 * the documented data format, never through code):
 *   - grid nx*ny*nz cells, box [0,lx]x[0,ly]x[0,lz]; x and z periodic,
 *     y bounded by walls at y=0 and y=ly (the paper's x3, Section 2).
 *   - u on x-faces  (i*dx, (j+.5)*dy, (k+.5)*dz), j in [0,ny)
 *     v on y-faces  ((i+.5)*dx, j*dy, (k+.5)*dz), j in [0,ny], walls j=0,ny
 *     w on z-faces  ((i+.5)*dx, (j+.5)*dy, k*dz), j in [0,ny)
 *     p, phi at cell centres.  Arrays are [k][j][i], i fastest; v has ny+1
 *     planes.
 *   - Compile with -ffp-contract=off: the tagging predicates must round
 *     exactly as written (no fused multiply-add).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nx, ny, nz;
  int ybc;              /* 0: no-slip walls, 1: free-slip walls (tests) */
  double lx, ly, lz;
  double dx, dy, dz;
  const double* yf;     /* ny + 1 wall-normal face positions (yf[0] = 0, yf[ny] = ly) of a
                           non-uniform grid (Section 2: variable cell size in the wall-normal
                           direction), or NULL for the uniform spacing dy */
} orc_grid;

/* ------------------------------------------------------------------ */
/* grid helpers                                                        */
/* ------------------------------------------------------------------ */

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops from now on (the timing of the oracle on one
 * core); n < 1 leaves the setting unchanged. */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void orc_grid_init(orc_grid* g, int nx, int ny, int nz, double lx, double ly, double lz, int ybc) {
  g->nx = nx; g->ny = ny; g->nz = nz; g->ybc = ybc;
  g->lx = lx; g->ly = ly; g->lz = lz;
  g->dx = lx / (double)nx;
  g->dy = ly / (double)ny;
  g->dz = lz / (double)nz;
  g->yf = NULL;
}

/* Wall-normal spacings (Section 2, variable cell size in the wall-normal
 * direction).  Cell j spans [yf[j], yf[j+1]]: height dyc(j), centre at the
 * midpoint.  Across face j the centres are dyf(j) apart; at the walls the
 * distance is to the mirror image of the first or last centre, so
 * dyf(0) = dyc(0) and dyf(ny) = dyc(ny-1), where the wall ghost lives.
 * With yf == NULL both return the uniform dy. */
static double dyc(const orc_grid* g, long j) { return g->yf ? g->yf[j + 1] - g->yf[j] : g->dy; }
static double ycen(const orc_grid* g, long j) { return 0.5 * (g->yf[j] + g->yf[j + 1]); }
static double dyf(const orc_grid* g, long j) {
  if (!g->yf) return g->dy;
  if (j <= 0) return dyc(g, 0);
  if (j >= g->ny) return dyc(g, g->ny - 1);
  return ycen(g, j) - ycen(g, j - 1);
}

/* number of y-planes stored for component c (v carries both wall planes) */
static int planes(const orc_grid* g, int c) { return c == 1 ? g->ny + 1 : g->ny; }

static long fidx(const orc_grid* g, int c, long i, long j, long k) {
  return (k * planes(g, c) + j) * (long)g->nx + i;
}

static long cidx(const orc_grid* g, long i, long j, long k) {
  return (k * g->ny + j) * (long)g->nx + i;
}

static long wrap(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

/* Staggered node position of component c with (possibly unwrapped) lattice
 * indices (i,j,k): Fig. problem_and_grid(b), Section 2. */
/* Wall-normal coordinate of lattice row j: cell centres (half = 1) or faces
 * (half = 0).  On the non-uniform grid a row beyond a wall is the mirror
 * image of the row inside it (where the wall ghosts of Section 2 live). */
static double ylat(const orc_grid* g, long j, int half) {
  if (!g->yf) return half ? ((double)j + 0.5) * g->dy : (double)j * g->dy;
  const long ny = g->ny;
  if (half) {
    if (j < 0) return 2.0 * g->yf[0] - ycen(g, -1 - j);
    if (j >= ny) return 2.0 * g->yf[ny] - ycen(g, 2 * ny - 1 - j);
    return ycen(g, j);
  }
  if (j < 0) return 2.0 * g->yf[0] - g->yf[-j];
  if (j > ny) return 2.0 * g->yf[ny] - g->yf[2 * ny - j];
  return g->yf[j];
}

static void node_xyz(const orc_grid* g, int c, long i, long j, long k, double x[3]) {
  x[0] = (c == 0) ? (double)i * g->dx : ((double)i + 0.5) * g->dx;
  x[1] = ylat(g, j, c != 1);
  x[2] = (c == 2) ? (double)k * g->dz : ((double)k + 0.5) * g->dz;
}

/* Wall-normal size of the local Eulerian cell of a node of component c in
 * row j (Algorithm 1, Section 3.1): the cell height for u and w (cell
 * centres), the distance between the centres on either side for v (faces). */
static double hy_of(const orc_grid* g, int c, long j) {
  if (!g->yf) return g->dy;
  return c == 1 ? dyf(g, j) : dyc(g, j);
}

/* Squared diagonal of the local Eulerian cell of that node. */
static double diag2_at(const orc_grid* g, int c, long j) {
  const double hy = hy_of(g, c, j);
  return (g->dx * g->dx + hy * hy) + g->dz * g->dz;
}

/* Offsets of component c's lattice in units of the spacing. */
static void node_offset(int c, double off[3]) {
  off[0] = (c == 0) ? 0.0 : 0.5;
  off[1] = (c == 1) ? 0.0 : 0.5;
  off[2] = (c == 2) ? 0.0 : 0.5;
}

/* Range of y indices that hold unknowns of component c. */
static void jrange(const orc_grid* g, int c, long* jlo, long* jhi) {
  if (c == 1) { *jlo = 1; *jhi = g->ny - 1; }
  else        { *jlo = 0; *jhi = g->ny - 1; }
}

static double dot3(const double a[3], const double b[3]) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* ------------------------------------------------------------------ */
/* Closest point on a triangle (Algorithm 1, step "closest point",     */
/* which cites Ericson 2004).  Voronoi-region classification of p      */
/* against the vertex, edge and face regions of triangle (a,b,c), with  */
/* the textbook quantities: the six scalar products of the edge vectors */
/* with p - a, p - b and p - c, each formed from its own difference     */
/* vector, and the edge and face parameters as the quotients of those   */
/* products (t = d1 / (d1 - d3), ..., s = 1 / (va + vb + vc)).          */
/* Returns X and its barycentric weights w (w[0]+w[1]+w[2]=1).         */
/* ------------------------------------------------------------------ */
void orc_closest_point(const double p[3], const double a[3], const double b[3], const double c[3],
                       double X[3], double w[3]) {
  double ab[3], ac[3], ap[3], bp[3], cp[3];
  for (int d = 0; d < 3; ++d) {
    ab[d] = b[d] - a[d];
    ac[d] = c[d] - a[d];
    ap[d] = p[d] - a[d];
  }
  const double d1 = dot3(ab, ap);
  const double d2 = dot3(ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) {                         /* vertex a region */
    for (int d = 0; d < 3; ++d) X[d] = a[d];
    w[0] = 1.0; w[1] = 0.0; w[2] = 0.0;
    return;
  }
  for (int d = 0; d < 3; ++d) bp[d] = p[d] - b[d];
  const double d3 = dot3(ab, bp);
  const double d4 = dot3(ac, bp);
  if (d3 >= 0.0 && d4 <= d3) {                          /* vertex b region */
    for (int d = 0; d < 3; ++d) X[d] = b[d];
    w[0] = 0.0; w[1] = 1.0; w[2] = 0.0;
    return;
  }
  const double vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {           /* edge ab region */
    const double t = d1 / (d1 - d3);
    for (int d = 0; d < 3; ++d) X[d] = a[d] + t * ab[d];
    w[0] = 1.0 - t; w[1] = t; w[2] = 0.0;
    return;
  }
  for (int d = 0; d < 3; ++d) cp[d] = p[d] - c[d];
  const double d5 = dot3(ab, cp);
  const double d6 = dot3(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) {                          /* vertex c region */
    for (int d = 0; d < 3; ++d) X[d] = c[d];
    w[0] = 0.0; w[1] = 0.0; w[2] = 1.0;
    return;
  }
  const double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {           /* edge ac region */
    const double t = d2 / (d2 - d6);
    for (int d = 0; d < 3; ++d) X[d] = a[d] + t * ac[d];
    w[0] = 1.0 - t; w[1] = 0.0; w[2] = t;
    return;
  }
  const double va = d3 * d6 - d5 * d4;
  if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) { /* edge bc region */
    const double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    for (int d = 0; d < 3; ++d) X[d] = b[d] + t * (c[d] - b[d]);
    w[0] = 0.0; w[1] = 1.0 - t; w[2] = t;
    return;
  }
  const double s = 1.0 / ((va + vb) + vc);              /* face region */
  const double v = vb * s;
  const double u = vc * s;
  for (int d = 0; d < 3; ++d) X[d] = (a[d] + ab[d] * v) + ac[d] * u;
  w[0] = (1.0 - v) - u; w[1] = v; w[2] = u;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1, body of the inner loop: decide whether node x (lattice  */
/* indices i,j,k of component c, unwrapped) is a forcing node for the   */
/* triangle (a,b,c3).  Returns 1 and |N|^2 if so.                       */
/*   |N| <= diagonal of the local cell (compared squared);             */
/*   forcing iff some scalar product N . (x^{k,n} - X) < 0 over the six */
/*   lattice neighbours x^{k,n}.  A node lying on the surface (N = 0)   */
/*   has no defined side and is tagged, with alpha = 0 in Eq. new_IB.  */
/* ------------------------------------------------------------------ */
static int tag_test(const orc_grid* g, int c, long i, long j, long k, const double x[3],
                    const double* a, const double* b, const double* c3, double diag2, double* n2_out) {
  double X[3], w[3], N[3];
  orc_closest_point(x, a, b, c3, X, w);
  for (int d = 0; d < 3; ++d) N[d] = x[d] - X[d];
  double n2 = dot3(N, N);
  if (!(n2 <= diag2)) return 0;
  *n2_out = n2;
  if (n2 == 0.0) return 1;
  for (int d = 0; d < 3; ++d) {
    for (int s = -1; s <= 1; s += 2) {
      long ni = i + (d == 0 ? s : 0);
      long nj = j + (d == 1 ? s : 0);
      long nk = k + (d == 2 ? s : 0);
      double xn[3], vn[3];
      node_xyz(g, c, ni, nj, nk, xn);
      for (int e = 0; e < 3; ++e) vn[e] = xn[e] - X[e];
      if (dot3(N, vn) < 0.0) return 1;
    }
  }
  return 0;
}

static void tri_vertices(const double* xyz, const int* tri, long t, const double** a, const double** b,
                         const double** c) {
  *a = xyz + 3 * (long)tri[3 * t + 0];
  *b = xyz + 3 * (long)tri[3 * t + 1];
  *c = xyz + 3 * (long)tri[3 * t + 2];
}

static double diag2_of(const orc_grid* g) { return diag2_at(g, 0, 0); }

/* Owner rule when several triangles tag the same node: the one with the
 * smallest |N|^2, ties to the smallest triangle index. */
static void claim(int32_t* owner, double* d2, long idx, int32_t t, double n2) {
  if (owner[idx] < 0 || n2 < d2[idx] || (n2 == d2[idx] && t < owner[idx])) {
    owner[idx] = t;
    d2[idx] = n2;
  }
}

/* Algorithm 1 as printed: loop over triangles, build the Cartesian box
 * min - dx < x < max + dx (strict), visit the Eulerian points of component c
 * inside it, and classify each.  Indices that leave the box in x or z wrap
 * periodically (the point keeps its unwrapped coordinate).  Only nodes whose
 * wrapped x index lies in [i0, i0 + ni) are recorded, in arrays laid out
 * [k][j][i - i0] (ni = nx: the whole component).  owner[] must be -1 on
 * entry; d2[] is scratch of the same size. */
static void tag_alg1_window(const orc_grid* g, int c, const double* xyz, int ntri, const int* tri, long i0,
                            long ni, int32_t* owner, double* d2) {
  double off[3], del[3] = {g->dx, g->dy, g->dz};
  node_offset(c, off);
  long jlo, jhi;
  jrange(g, c, &jlo, &jhi);
  for (long t = 0; t < ntri; ++t) {
    const double *a, *b, *c3;
    tri_vertices(xyz, tri, t, &a, &b, &c3);
    double lo[3], hi[3];
    long ilo[3], ihi[3];
    for (int d = 0; d < 3; ++d) {
      double mn = fmin(a[d], fmin(b[d], c3[d]));
      double mx = fmax(a[d], fmax(b[d], c3[d]));
      lo[d] = mn - del[d];
      hi[d] = mx + del[d];
      ilo[d] = (long)floor(lo[d] / del[d] - off[d]) - 1;
      ihi[d] = (long)ceil(hi[d] / del[d] - off[d]) + 1;
    }
    if (g->yf) {
      /* non-uniform rows: the box margin in y is the node's own cell size,
       * so every row is visited and the predicate below decides */
      ilo[1] = jlo;
      ihi[1] = jhi;
    }
    if (ilo[1] < jlo) ilo[1] = jlo;
    if (ihi[1] > jhi) ihi[1] = jhi;
    for (long k = ilo[2]; k <= ihi[2]; ++k)
      for (long j = ilo[1]; j <= ihi[1]; ++j) {
        if (g->yf) {
          const double hy = hy_of(g, c, j);
          lo[1] = fmin(a[1], fmin(b[1], c3[1])) - hy;
          hi[1] = fmax(a[1], fmax(b[1], c3[1])) + hy;
        }
        for (long i = ilo[0]; i <= ihi[0]; ++i) {
          double x[3];
          node_xyz(g, c, i, j, k, x);
          int inside = 1;
          for (int d = 0; d < 3; ++d)
            if (!(lo[d] < x[d] && x[d] < hi[d])) inside = 0;
          if (!inside) continue;
          const long iw = wrap(i, g->nx) - i0;
          if (iw < 0 || iw >= ni) continue;
          double n2;
          if (tag_test(g, c, i, j, k, x, a, b, c3, diag2_at(g, c, j), &n2)) {
            long planes = (c == 1) ? g->ny + 1 : g->ny;
            long idx = (wrap(k, g->nz) * planes + j) * ni + iw;
            claim(owner, d2, idx, (int32_t)t, n2);
          }
        }
      }
  }
}

void orc_tag_alg1(const orc_grid* g, int c, const double* xyz, int ntri, const int* tri,
                  int32_t* owner, double* d2) {
  tag_alg1_window(g, c, xyz, ntri, tri, 0, g->nx, owner, d2);
}

/* Algorithm 1 restricted to the nodes with x index in [i0, i0 + ni): the
 * exact owners of a slab of a grid too large to tag whole. */
void orc_tag_alg1_window(const orc_grid* g, int c, const double* xyz, int ntri, const int* tri, long i0, long ni,
                         int32_t* owner, double* d2) {
  tag_alg1_window(g, c, xyz, ntri, tri, i0, ni, owner, d2);
}

/* Brute force counterpart of Algorithm 1: every node of component c (and
 * its periodic images one box away in x and z) against every triangle, with
 * the bounding box applied as a predicate.  Tiny grids only. */
void orc_tag_brute(const orc_grid* g, int c, const double* xyz, int ntri, const int* tri,
                   int32_t* owner, double* d2) {
  long jlo, jhi;
  jrange(g, c, &jlo, &jhi);
  for (long k = 0; k < g->nz; ++k)
    for (long j = jlo; j <= jhi; ++j)
      for (long i = 0; i < g->nx; ++i) {
        /* the box margin and the diagonal are those of the node's local cell */
        const double del[3] = {g->dx, hy_of(g, c, j), g->dz};
        const double diag2 = diag2_at(g, c, j);
        long idx = fidx(g, c, i, j, k);
        for (int mk = -1; mk <= 1; ++mk)
          for (int mi = -1; mi <= 1; ++mi) {
            long ii = i + mi * (long)g->nx, kk = k + mk * (long)g->nz;
            double x[3];
            node_xyz(g, c, ii, j, kk, x);
            for (long t = 0; t < ntri; ++t) {
              const double *a, *b, *c3;
              tri_vertices(xyz, tri, t, &a, &b, &c3);
              int inside = 1;
              for (int d = 0; d < 3; ++d) {
                double mn = fmin(a[d], fmin(b[d], c3[d]));
                double mx = fmax(a[d], fmax(b[d], c3[d]));
                if (!((mn - del[d]) < x[d] && x[d] < (mx + del[d]))) inside = 0;
              }
              if (!inside) continue;
              double n2;
              if (tag_test(g, c, ii, j, kk, x, a, b, c3, diag2, &n2)) claim(owner, d2, idx, (int32_t)t, n2);
            }
          }
      }
}

/* ------------------------------------------------------------------ */
/* Trilinear interpolation of component c at point P from the 8        */
/* surrounding nodes of the same staggered lattice (Section 3.1, the   */
/* interpolation of u^e).  x and z wrap; in y the 8 nodes must lie in  */
/* the stored planes (u,w: 0..ny-1, v: 0..ny incl. the wall values),    */
/* otherwise returns -1 (probe left the domain).                        */
/* ------------------------------------------------------------------ */
static int trilinear(const orc_grid* g, int c, const double* f, const double P[3], double* out) {
  double off[3], del[3] = {g->dx, g->dy, g->dz};
  node_offset(c, off);
  long i0[3];
  double t[3];
  for (int d = 0; d < 3; ++d) {
    double s = P[d] / del[d] - off[d];
    double fl = floor(s);
    i0[d] = (long)fl;
    t[d] = s - fl;
  }
  long jmax = planes(g, c) - 1;
  if (g->yf) {
    /* non-uniform rows: the bracketing pair by bisection, the weight from
     * the two row coordinates */
    const int half = c != 1;
    if (!(ylat(g, 0, half) <= P[1] && P[1] < ylat(g, jmax, half))) return -1;
    long ja = 0, jb = jmax;   /* ylat(ja) <= P[1] < ylat(jb) */
    while (jb - ja > 1) {
      long jm = (ja + jb) / 2;
      if (ylat(g, jm, half) <= P[1]) ja = jm; else jb = jm;
    }
    i0[1] = ja;
    t[1] = (P[1] - ylat(g, ja, half)) / (ylat(g, ja + 1, half) - ylat(g, ja, half));
  }
  if (i0[1] < 0 || i0[1] + 1 > jmax) return -1;
  double acc = 0.0;
  for (int dk = 0; dk <= 1; ++dk)
    for (int dj = 0; dj <= 1; ++dj)
      for (int di = 0; di <= 1; ++di) {
        double wgt = (di ? t[0] : 1.0 - t[0]) * (dj ? t[1] : 1.0 - t[1]) * (dk ? t[2] : 1.0 - t[2]);
        long ii = wrap(i0[0] + di, g->nx), jj = i0[1] + dj, kk = wrap(i0[2] + dk, g->nz);
        acc += wgt * f[fidx(g, c, ii, jj, kk)];
      }
  *out = acc;
  return 0;
}

/* Lattice position of stored node (i,j,k) taken at the periodic image
 * nearest to the owning triangle's centroid (the image Algorithm 1 visited). */
static void node_near(const orc_grid* g, int c, long i, long j, long k, const double* a, const double* b,
                      const double* c3, double x[3]) {
  double cen[3];
  for (int d = 0; d < 3; ++d) cen[d] = (a[d] + b[d] + c3[d]) / 3.0;
  node_xyz(g, c, i, j, k, x);
  long mi = lround((cen[0] - x[0]) / g->lx);
  long mk = lround((cen[2] - x[2]) / g->lz);
  node_xyz(g, c, i + mi * (long)g->nx, j, k + mk * (long)g->nz, x);
}

/* ------------------------------------------------------------------ */
/* Two-sided IB forcing, Eqs. probe and new_IB: for every forcing node */
/* x^f of component c, X^f = closest point on its triangle, N = x^f-X, */
/* n = N/|N|, x^e = X^f + h n, u^e trilinear from the snapshot `src`,  */
/* U = wall velocity at X^f (barycentric from the vertex velocities),  */
/* alpha = |N|/h, u^f = (1-alpha) U + alpha u^e.  Writes u^f into dst  */
/* at the forcing nodes only.  Returns the number of probes that left  */
/* the domain (0 on success).  h is the probe length of a uniform      */
/* grid; on a non-uniform wall-normal grid every node takes twice the   */
/* diagonal of its own cell (Section 3.1) and the argument is not read. */
/* ------------------------------------------------------------------ */
int orc_force(const orc_grid* g, int c, const double* src, double* dst, const int32_t* owner,
              const double* xyz, const double* vel, const int* tri, double h) {
  long n = (long)g->nz * planes(g, c) * g->nx;
  int bad = 0;
  for (long idx = 0; idx < n; ++idx) {
    int32_t t = owner[idx];
    if (t < 0) continue;
    long i = idx % g->nx, j = (idx / g->nx) % planes(g, c), k = idx / ((long)g->nx * planes(g, c));
    const double *a, *b, *c3;
    tri_vertices(xyz, tri, t, &a, &b, &c3);
    double x[3], X[3], w[3], N[3];
    node_near(g, c, i, j, k, a, b, c3, x);
    orc_closest_point(x, a, b, c3, X, w);
    for (int d = 0; d < 3; ++d) N[d] = x[d] - X[d];
    double U = w[0] * vel[3 * (long)tri[3 * t + 0] + c] + w[1] * vel[3 * (long)tri[3 * t + 1] + c] +
               w[2] * vel[3 * (long)tri[3 * t + 2] + c];
    double n2 = dot3(N, N);
    if (n2 == 0.0) { dst[idx] = U; continue; }
    if (g->yf) h = 2.0 * sqrt(diag2_at(g, c, j));   /* twice the local diagonal */
    double nl = sqrt(n2);
    double xe[3];
    for (int d = 0; d < 3; ++d) xe[d] = X[d] + h * (N[d] / nl);
    double ue;
    if (trilinear(g, c, src, xe, &ue) != 0) { bad++; continue; }
    double alpha = nl / h;
    dst[idx] = (1.0 - alpha) * U + alpha * ue;
  }
  return bad;
}

/* ------------------------------------------------------------------ */
/* No-slip error on the forcing points of component c (Section 4.4,   */
/* heaving plate): the flow is interpolated on the surface with the     */
/* interpolator of Eq. new_IB, u_w = (u(x^f) - alpha u(x^e))/(1-alpha), */
/* eps = u_w - U.  Returns sum |eps| and the count through pointers.   */
/* h as in orc_force.                                                   */
/* ------------------------------------------------------------------ */
int orc_slip(const orc_grid* g, int c, const double* f, const int32_t* owner, const double* xyz,
             const double* vel, const int* tri, double h, double* sum_abs, long* count) {
  long n = (long)g->nz * planes(g, c) * g->nx;
  double s = 0.0;
  long cnt = 0;
  int bad = 0;
  for (long idx = 0; idx < n; ++idx) {
    int32_t t = owner[idx];
    if (t < 0) continue;
    long i = idx % g->nx, j = (idx / g->nx) % planes(g, c), k = idx / ((long)g->nx * planes(g, c));
    const double *a, *b, *c3;
    tri_vertices(xyz, tri, t, &a, &b, &c3);
    double x[3], X[3], w[3], N[3];
    node_near(g, c, i, j, k, a, b, c3, x);
    orc_closest_point(x, a, b, c3, X, w);
    for (int d = 0; d < 3; ++d) N[d] = x[d] - X[d];
    double U = w[0] * vel[3 * (long)tri[3 * t + 0] + c] + w[1] * vel[3 * (long)tri[3 * t + 1] + c] +
               w[2] * vel[3 * (long)tri[3 * t + 2] + c];
    double n2 = dot3(N, N);
    double uw;
    if (n2 == 0.0) {
      uw = f[idx];
    } else {
      if (g->yf) h = 2.0 * sqrt(diag2_at(g, c, j));   /* twice the local diagonal */
      double nl = sqrt(n2);
      double xe[3];
      for (int d = 0; d < 3; ++d) xe[d] = X[d] + h * (N[d] / nl);
      double ue;
      if (trilinear(g, c, f, xe, &ue) != 0) { bad++; continue; }
      double alpha = nl / h;
      uw = (f[idx] - alpha * ue) / (1.0 - alpha);
    }
    s += fabs(uw - U);
    cnt++;
  }
  *sum_abs = s;
  *count = cnt;
  return bad;
}

/* ------------------------------------------------------------------ */
/* Explicit part of Eq. NS_prov on the fluid nodes:                    */
/*   R = dt [ gamma H^s + rho H^{s-1} - alpha G p^s + alpha/Re L u^s   */
/*            + alpha f ]                                               */
/* (the CN half alpha/(2Re) L(uhat+u^s) written in delta form adds     */
/*  alpha/Re L u^s here; the other half is the implicit operator).      */
/* H is the conservative non-linear term -div(u u) on the staggered     */
/* grid with arithmetic face/edge averages (Section 2, "conservative    */
/* form", second-order centred).  R = 0 on forcing nodes.  H is          */
/* returned on every node.  Hprev may be NULL when rho == 0.            */
/* Tangential wall condition: ghost u_{-1} = -u_0 (no-slip, wall at     */
/* rest) or u_{-1} = u_0 (free-slip); v = 0 on the walls.               */
/* ------------------------------------------------------------------ */
void orc_rhs(const orc_grid* g, const double* u, const double* v, const double* w, const double* p,
             const double* Hu_prev, const double* Hv_prev, const double* Hw_prev,
             const int32_t* own_u, const int32_t* own_v, const int32_t* own_w,
             double gam, double rho, double alp, double dt, double re, const double fb[3],
             double* Ru, double* Rv, double* Rw, double* Hu, double* Hv, double* Hw) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const double dx = g->dx, dy = g->dy, dz = g->dz;
  const double gs = (g->ybc == 0) ? -1.0 : 1.0; /* ghost sign for tangential components */
#define U(i, j, k) u[fidx(g, 0, wrap(i, nx), j, wrap(k, nz))]
#define V(i, j, k) v[fidx(g, 1, wrap(i, nx), j, wrap(k, nz))]
#define W(i, j, k) w[fidx(g, 2, wrap(i, nx), j, wrap(k, nz))]
#define P(i, j, k) p[cidx(g, wrap(i, nx), j, wrap(k, nz))]
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        /* wall-normal spacings of this row: cell height, centre distances below and above */
        const int nun = g->yf != NULL;
        const double hc = dyc(g, j), hs = dyf(g, j), hn = dyf(g, j + 1);
        /* ---- u at (i dx, (j+.5) dy, (k+.5) dz) ---- */
        {
          double uc_p = 0.5 * (U(i, j, k) + U(i + 1, j, k));
          double uc_m = 0.5 * (U(i - 1, j, k) + U(i, j, k));
          double duu = (uc_p * uc_p - uc_m * uc_m) / dx;
          double vt = 0.5 * (V(i - 1, j + 1, k) + V(i, j + 1, k));
          double ut = (j + 1 < ny) ? 0.5 * (U(i, j, k) + U(i, j + 1, k)) : 0.0;
          double vb = 0.5 * (V(i - 1, j, k) + V(i, j, k));
          double ub = (j > 0) ? 0.5 * (U(i, j - 1, k) + U(i, j, k)) : 0.0;
          double dvu = (vt * ut - vb * ub) / hc;
          double wf = 0.5 * (W(i - 1, j, k + 1) + W(i, j, k + 1));
          double uf = 0.5 * (U(i, j, k) + U(i, j, k + 1));
          double wb = 0.5 * (W(i - 1, j, k) + W(i, j, k));
          double ubk = 0.5 * (U(i, j, k - 1) + U(i, j, k));
          double dwu = (wf * uf - wb * ubk) / dz;
          double H = -(duu + dvu + dwu);
          double c0 = U(i, j, k);
          double ujm = (j > 0) ? U(i, j - 1, k) : gs * c0;
          double ujp = (j + 1 < ny) ? U(i, j + 1, k) : gs * c0;
          double Ly = nun ? ((ujp - c0) / hn - (c0 - ujm) / hs) / hc : (ujp - 2.0 * c0 + ujm) / (dy * dy);
          double L = (U(i + 1, j, k) - 2.0 * c0 + U(i - 1, j, k)) / (dx * dx) + Ly +
                     (U(i, j, k + 1) - 2.0 * c0 + U(i, j, k - 1)) / (dz * dz);
          double G = (P(i, j, k) - P(i - 1, j, k)) / dx;
          long id = fidx(g, 0, i, j, k);
          double r = gam * H - alp * G + (alp / re) * L + alp * fb[0];
          if (rho != 0.0) r += rho * Hu_prev[id];
          Hu[id] = H;
          Ru[id] = own_u[id] >= 0 ? 0.0 : dt * r;
        }
        /* ---- w at ((i+.5) dx, (j+.5) dy, k dz) ---- */
        {
          double ur = 0.5 * (U(i + 1, j, k - 1) + U(i + 1, j, k));
          double wr = 0.5 * (W(i, j, k) + W(i + 1, j, k));
          double ul = 0.5 * (U(i, j, k - 1) + U(i, j, k));
          double wl = 0.5 * (W(i - 1, j, k) + W(i, j, k));
          double duw = (ur * wr - ul * wl) / dx;
          double vt = 0.5 * (V(i, j + 1, k - 1) + V(i, j + 1, k));
          double wt = (j + 1 < ny) ? 0.5 * (W(i, j, k) + W(i, j + 1, k)) : 0.0;
          double vb = 0.5 * (V(i, j, k - 1) + V(i, j, k));
          double wbj = (j > 0) ? 0.5 * (W(i, j - 1, k) + W(i, j, k)) : 0.0;
          double dvw = (vt * wt - vb * wbj) / hc;
          double wc_p = 0.5 * (W(i, j, k) + W(i, j, k + 1));
          double wc_m = 0.5 * (W(i, j, k - 1) + W(i, j, k));
          double dww = (wc_p * wc_p - wc_m * wc_m) / dz;
          double H = -(duw + dvw + dww);
          double c0 = W(i, j, k);
          double wjm = (j > 0) ? W(i, j - 1, k) : gs * c0;
          double wjp = (j + 1 < ny) ? W(i, j + 1, k) : gs * c0;
          double Ly = nun ? ((wjp - c0) / hn - (c0 - wjm) / hs) / hc : (wjp - 2.0 * c0 + wjm) / (dy * dy);
          double L = (W(i + 1, j, k) - 2.0 * c0 + W(i - 1, j, k)) / (dx * dx) + Ly +
                     (W(i, j, k + 1) - 2.0 * c0 + W(i, j, k - 1)) / (dz * dz);
          double G = (P(i, j, k) - P(i, j, k - 1)) / dz;
          long id = fidx(g, 2, i, j, k);
          double r = gam * H - alp * G + (alp / re) * L + alp * fb[2];
          if (rho != 0.0) r += rho * Hw_prev[id];
          Hw[id] = H;
          Rw[id] = own_w[id] >= 0 ? 0.0 : dt * r;
        }
        /* ---- v at ((i+.5) dx, j dy, (k+.5) dz), interior faces only ---- */
        if (j >= 1) {
          double ur = 0.5 * (U(i + 1, j - 1, k) + U(i + 1, j, k));
          double vr = 0.5 * (V(i, j, k) + V(i + 1, j, k));
          double ul = 0.5 * (U(i, j - 1, k) + U(i, j, k));
          double vl = 0.5 * (V(i - 1, j, k) + V(i, j, k));
          double duv = (ur * vr - ul * vl) / dx;
          double vc_p = 0.5 * (V(i, j, k) + V(i, j + 1, k));
          double vc_m = 0.5 * (V(i, j - 1, k) + V(i, j, k));
          double dvv = (vc_p * vc_p - vc_m * vc_m) / hs;
          double wf = 0.5 * (W(i, j - 1, k + 1) + W(i, j, k + 1));
          double vf = 0.5 * (V(i, j, k) + V(i, j, k + 1));
          double wb = 0.5 * (W(i, j - 1, k) + W(i, j, k));
          double vbk = 0.5 * (V(i, j, k - 1) + V(i, j, k));
          double dwv = (wf * vf - wb * vbk) / dz;
          double H = -(duv + dvv + dwv);
          double c0 = V(i, j, k);
          double Ly = nun ? ((V(i, j + 1, k) - c0) / hc - (c0 - V(i, j - 1, k)) / dyc(g, j - 1)) / hs
                          : (V(i, j + 1, k) - 2.0 * c0 + V(i, j - 1, k)) / (dy * dy);
          double L = (V(i + 1, j, k) - 2.0 * c0 + V(i - 1, j, k)) / (dx * dx) + Ly +
                     (V(i, j, k + 1) - 2.0 * c0 + V(i, j, k - 1)) / (dz * dz);
          double G = (P(i, j, k) - P(i, j - 1, k)) / hs;
          long id = fidx(g, 1, i, j, k);
          double r = gam * H - alp * G + (alp / re) * L + alp * fb[1];
          if (rho != 0.0) r += rho * Hv_prev[id];
          Hv[id] = H;
          Rv[id] = own_v[id] >= 0 ? 0.0 : dt * r;
        }
      }
  /* wall planes of v carry no unknown */
  for (long k = 0; k < nz; ++k)
    for (long i = 0; i < nx; ++i) {
      Rv[fidx(g, 1, i, 0, k)] = 0.0;  Hv[fidx(g, 1, i, 0, k)] = 0.0;
      Rv[fidx(g, 1, i, ny, k)] = 0.0; Hv[fidx(g, 1, i, ny, k)] = 0.0;
    }
#undef U
#undef V
#undef W
#undef P
}

/* ------------------------------------------------------------------ */
/* Tridiagonal solvers (Thomas algorithm, and its periodic variant by   */
/* the Sherman-Morrison correction).  a = sub, b = diag, c = super.     */
/* ------------------------------------------------------------------ */
static void thomas(int n, const double* a, const double* b, const double* c, double* x, double* cw) {
  /* solves in place: x holds the right-hand side on entry */
  cw[0] = c[0] / b[0];
  x[0] = x[0] / b[0];
  for (int i = 1; i < n; ++i) {
    double den = b[i] - a[i] * cw[i - 1];
    cw[i] = c[i] / den;
    x[i] = (x[i] - a[i] * x[i - 1]) / den;
  }
  for (int i = n - 2; i >= 0; --i) x[i] = x[i] - cw[i] * x[i + 1];
}

/* periodic system: a[0] couples row 0 to x[n-1], c[n-1] couples row n-1 to x[0] */
static void thomas_periodic(int n, const double* a, const double* b, const double* c, double* x,
                            double* bb, double* z, double* cw) {
  double gam = -b[0];
  for (int i = 0; i < n; ++i) bb[i] = b[i];
  bb[0] = b[0] - gam;
  bb[n - 1] = b[n - 1] - c[n - 1] * a[0] / gam;
  thomas(n, a, bb, c, x, cw);
  for (int i = 0; i < n; ++i) z[i] = 0.0;
  z[0] = gam;
  z[n - 1] = c[n - 1];
  thomas(n, a, bb, c, z, cw);
  double fact = (x[0] + a[0] * x[n - 1] / gam) / (1.0 + z[0] + a[0] * z[n - 1] / gam);
  for (int i = 0; i < n; ++i) x[i] -= fact * z[i];
}

/* ------------------------------------------------------------------ */
/* Approximate factorisation of the CN operator (Section 2, after Eq.  */
/* NS_prov): (1 - beta L_x)(1 - beta L_z)(1 - beta L_y) du = R, solved */
/* one direction at a time, x first, then z, then y; beta =            */
/* alpha dt / (2 Re).  Forcing nodes are identity rows (the equation is */
/* solved on all points but the forcing points).  x and z periodic; in  */
/* y the tangential components use the wall ghost of orc_rhs and v has  */
/* du = 0 on the wall planes.  In-place on `f` (component c).           */
/* ------------------------------------------------------------------ */
void orc_sweep(const orc_grid* g, int c, int dir, double* f, const int32_t* owner, double beta) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const long pl = planes(g, c);
  if (dir == 0 || dir == 2) {
    const int n = dir == 0 ? nx : nz;
    const double dd = dir == 0 ? g->dx : g->dz;
    const double off = beta / (dd * dd);
    const int nl1 = dir == 0 ? (int)pl : (int)pl;   /* j planes */
    const int nl2 = dir == 0 ? nz : nx;
#pragma omp parallel for schedule(static)
    for (int l2 = 0; l2 < nl2; ++l2) {
      double *a = malloc(sizeof(double) * n * 7), *b = a + n, *cc = b + n, *x = cc + n, *bb = x + n, *z = bb + n,
             *cw = z + n;
      for (int j = 0; j < nl1; ++j) {
        if (c == 1 && (j == 0 || j == ny)) continue;
        for (int m = 0; m < n; ++m) {
          long id = dir == 0 ? fidx(g, c, m, j, l2) : fidx(g, c, l2, j, m);
          if (owner[id] >= 0) { a[m] = 0.0; b[m] = 1.0; cc[m] = 0.0; }
          else { a[m] = -off; b[m] = 1.0 + 2.0 * off; cc[m] = -off; }
          x[m] = f[id];
        }
        thomas_periodic(n, a, b, cc, x, bb, z, cw);
        for (int m = 0; m < n; ++m) {
          long id = dir == 0 ? fidx(g, c, m, j, l2) : fidx(g, c, l2, j, m);
          f[id] = x[m];
        }
      }
      free(a);
    }
  } else if (g->yf) {
    /* non-uniform wall-normal spacing: the coefficients of the y part of
     * the Laplacian of orc_rhs, row by row */
    const double gs = (g->ybc == 0) ? -1.0 : 1.0;
    const int j0 = (c == 1) ? 1 : 0, n = ny - j0;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
      double *a = malloc(sizeof(double) * n * 5), *b = a + n, *cc = b + n, *x = cc + n, *cw = x + n;
      for (int i = 0; i < nx; ++i) {
        for (int m = 0; m < n; ++m) {
          const long j = j0 + m;
          long id = fidx(g, c, i, j, k);
          if (owner[id] >= 0) { a[m] = 0.0; b[m] = 1.0; cc[m] = 0.0; }
          else if (c != 1) {
            const double sb = beta / (dyc(g, j) * dyf(g, j)), sn = beta / (dyc(g, j) * dyf(g, j + 1));
            a[m] = -sb; b[m] = 1.0 + sb + sn; cc[m] = -sn;
            /* ghost du_{-1} = gs du_0 at the walls folds into the diagonal */
            if (m == 0) { b[m] -= gs * sb; a[m] = 0.0; }
            if (m == n - 1) { b[m] -= gs * sn; cc[m] = 0.0; }
          } else {
            const double sb = beta / (dyf(g, j) * dyc(g, j - 1)), sn = beta / (dyf(g, j) * dyc(g, j));
            a[m] = m == 0 ? 0.0 : -sb; b[m] = 1.0 + sb + sn; cc[m] = m == n - 1 ? 0.0 : -sn;
          }
          x[m] = f[id];
        }
        thomas(n, a, b, cc, x, cw);
        for (int m = 0; m < n; ++m) f[fidx(g, c, i, j0 + m, k)] = x[m];
      }
      free(a);
    }
  } else {
    const double off = beta / (g->dy * g->dy);
    const double gs = (g->ybc == 0) ? -1.0 : 1.0;
    const int j0 = (c == 1) ? 1 : 0, j1 = (c == 1) ? ny - 1 : ny - 1;
    const int n = j1 - j0 + 1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
      double *a = malloc(sizeof(double) * n * 5), *b = a + n, *cc = b + n, *x = cc + n, *cw = x + n;
      for (int i = 0; i < nx; ++i) {
        for (int m = 0; m < n; ++m) {
          long id = fidx(g, c, i, j0 + m, k);
          if (owner[id] >= 0) { a[m] = 0.0; b[m] = 1.0; cc[m] = 0.0; }
          else {
            a[m] = -off; b[m] = 1.0 + 2.0 * off; cc[m] = -off;
            if (c != 1) {
              /* ghost du_{-1} = gs du_0 folds into the diagonal of the wall rows */
              if (m == 0) { b[m] -= gs * off; a[m] = 0.0; }
              if (m == n - 1) { b[m] -= gs * off; cc[m] = 0.0; }
            } else {
              if (m == 0) a[m] = 0.0;
              if (m == n - 1) cc[m] = 0.0;
            }
          }
          x[m] = f[id];
        }
        thomas(n, a, b, cc, x, cw);
        for (int m = 0; m < n; ++m) f[fidx(g, c, i, j0 + m, k)] = x[m];
      }
      free(a);
    }
  }
}

/* ------------------------------------------------------------------ */
/* Discrete divergence (Eq. discrete_div) at every cell centre.        */
/* ------------------------------------------------------------------ */
void orc_divergence(const orc_grid* g, const double* u, const double* v, const double* w, double* div) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        double du = (u[fidx(g, 0, wrap(i + 1, nx), j, k)] - u[fidx(g, 0, i, j, k)]) / g->dx;
        double dv = (v[fidx(g, 1, i, j + 1, k)] - v[fidx(g, 1, i, j, k)]) / dyc(g, j);
        double dw = (w[fidx(g, 2, i, j, wrap(k + 1, nz))] - w[fidx(g, 2, i, j, k)]) / g->dz;
        div[cidx(g, i, j, k)] = du + dv + dw;
      }
}

/* Boundary-cell flags (Section 3.2, Fig. fluid_and_boundary_cells): a cell
 * is a boundary cell when every one of its six faces holds a forcing node
 * of the velocity component living there. */
void orc_boundary_cells(const orc_grid* g, const int32_t* own_u, const int32_t* own_v, const int32_t* own_w,
                        uint8_t* isb) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        int all = own_u[fidx(g, 0, i, j, k)] >= 0 && own_u[fidx(g, 0, wrap(i + 1, nx), j, k)] >= 0 &&
                  own_v[fidx(g, 1, i, j, k)] >= 0 && own_v[fidx(g, 1, i, j + 1, k)] >= 0 &&
                  own_w[fidx(g, 2, i, j, k)] >= 0 && own_w[fidx(g, 2, i, j, wrap(k + 1, nz))] >= 0;
        isb[cidx(g, i, j, k)] = (uint8_t)all;
      }
}

/* Consistent mass correction and right-hand side of Eq. elliptic_mod:
 *   q_B = D uhat on boundary cells (Eq. q_boundary),
 *   q_F = -(1/|C_F|) sum_{C_B} D uhat dV, uniform on fluid cells,
 *   rhs = (D uhat - q) / (alpha dt)  (zero on C_B by construction).
 * With use_q = 0, q = 0 everywhere (the standard Eq. elliptic).  Returns
 * q_F; A = sum_{C_B} D uhat dV and V_F = |C_F| through pointers.  The sums
 * run in plain index order. */
double orc_rhs_poisson(const orc_grid* g, const double* div, const uint8_t* isb, int use_q, double adt,
                       double* rhs, double* A_out, double* VF_out) {
  const long n = (long)g->nx * g->ny * g->nz;
  double A = 0.0, VF = 0.0;
  for (long id = 0; id < n; ++id) {
    const double dV = (g->dx * dyc(g, (id / g->nx) % g->ny)) * g->dz;   /* cell volume */
    if (isb[id]) A += div[id] * dV;
    else VF += dV;
  }
  double qF = (use_q && VF > 0.0) ? -A / VF : 0.0;
  for (long id = 0; id < n; ++id) {
    double q = use_q ? (isb[id] ? div[id] : qF) : 0.0;
    rhs[id] = (div[id] - q) / adt;
  }
  *A_out = A;
  *VF_out = VF;
  return qF;
}

/* Energy- and mass-conserving shape of q on the fluid cells (App. B,
 * the minimiser of the augmented Lagrangian with the mass and the inviscid
 * kinetic-energy constraints):
 *   q_F^k = (-A S2 + B S1)/C + (A S1 - B S0)/C (p^k - e^k),
 *   S_i = sum_{C_F} (p - e)^i dV, A = sum_{C_B} Du dV,
 *   B = sum_{C_B} (p - e) Du dV, C = S0 S2 - S1^2.
 * Readings: p is the pressure p^s of the sub-stage, e = |u|^2/2 with the
 * velocity averaged to the cell centre from the provisional field uhat
 * (whose divergence div[] is); q = Du on C_B (Eq. q_boundary).  When C
 * vanishes (p - e uniform on C_F) the energy constraint is a multiple of
 * the mass one and the uniform shape -A/S0 is returned.  q[] gets the
 * field, coef[] = {alpha, beta, A, B, S0, S1, S2}. */
void orc_q_energy(const orc_grid* g, const double* div, const uint8_t* isb, const double* p, const double* u,
                  const double* v, const double* w, double* q, double* coef) {
  const long nx = g->nx, ny = g->ny, nz = g->nz, n = nx * ny * nz;
  double* pe = malloc(sizeof(double) * n);
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        const long id = (k * ny + j) * nx + i;
        const long ip = (i + 1) % nx, kp = (k + 1) % nz;
        const double uc = 0.5 * (u[(k * ny + j) * nx + i] + u[(k * ny + j) * nx + ip]);
        const double vc = 0.5 * (v[(k * (ny + 1) + j) * nx + i] + v[(k * (ny + 1) + j + 1) * nx + i]);
        const double wc = 0.5 * (w[(k * ny + j) * nx + i] + w[(kp * ny + j) * nx + i]);
        const double e = 0.5 * (uc * uc + vc * vc + wc * wc);
        pe[id] = p[id] - e;
      }
  double S0 = 0.0, S1 = 0.0, S2 = 0.0, A = 0.0, B = 0.0;
  for (long id = 0; id < n; ++id) {
    const double dV = (g->dx * dyc(g, (id / nx) % ny)) * g->dz;   /* cell volume */
    if (isb[id]) {
      A += div[id] * dV;
      B += pe[id] * div[id] * dV;
    } else {
      S0 += dV;
      S1 += pe[id] * dV;
      S2 += pe[id] * pe[id] * dV;
    }
  }
  const double C = S0 * S2 - S1 * S1;
  double alpha, beta;
  if (S0 > 0.0 && C > 1e-14 * S0 * S2) {
    alpha = (-A * S2 + B * S1) / C;
    beta = (A * S1 - B * S0) / C;
  } else {
    alpha = S0 > 0.0 ? -A / S0 : 0.0;
    beta = 0.0;
  }
  for (long id = 0; id < n; ++id) q[id] = isb[id] ? div[id] : alpha + beta * pe[id];
  coef[0] = alpha; coef[1] = beta; coef[2] = A; coef[3] = B; coef[4] = S0; coef[5] = S1; coef[6] = S2;
  free(pe);
}

/* ------------------------------------------------------------------ */
/* Wall-normal solve of the Poisson equation per Fourier mode (Eq.     */
/* elliptic, solved with FFTs in x and z and the Thomas algorithm in   */
/* y).  spec is [kz][j][kx] complex (re,im interleaved), nkx = nx/2+1; */
/* in place.  Row j: (phi_{j+1} - 2 phi_j + phi_{j-1})/dy^2            */
/*   - (lx + lz) phi_j = r_j, homogeneous Neumann at both walls, with    */
/* lx = (2 - 2 cos(2 pi kx / nx))/dx^2 (modified wavenumber of the      */
/* second difference), lz likewise.  Mode (0,0) is singular: phi_0 is   */
/* pinned to 0 and the mean over j is then removed (zero-mean gauge).   */
/* ------------------------------------------------------------------ */
void orc_poisson_y(const orc_grid* g, double* spec) {
  const int nx = g->nx, ny = g->ny, nz = g->nz, nkx = nx / 2 + 1;
  const double pi = 3.14159265358979323846;
  const double idy2 = 1.0 / (g->dy * g->dy);
#pragma omp parallel for schedule(static)
  for (int kz = 0; kz < nz; ++kz) {
    double *a = malloc(sizeof(double) * ny * 6), *b = a + ny, *c = b + ny, *xr = c + ny, *xi = xr + ny,
           *cw = xi + ny;
    for (int kx = 0; kx < nkx; ++kx) {
      double lam = (2.0 - 2.0 * cos(2.0 * pi * kx / nx)) / (g->dx * g->dx) +
                   (2.0 - 2.0 * cos(2.0 * pi * kz / nz)) / (g->dz * g->dz);
      for (int j = 0; j < ny; ++j) {
        if (g->yf) {   /* non-uniform rows of L_c (zero flux through the walls) */
          a[j] = (j > 0) ? 1.0 / (dyc(g, j) * dyf(g, j)) : 0.0;
          c[j] = (j < ny - 1) ? 1.0 / (dyc(g, j) * dyf(g, j + 1)) : 0.0;
        } else {
          a[j] = (j > 0) ? idy2 : 0.0;
          c[j] = (j < ny - 1) ? idy2 : 0.0;
        }
        b[j] = -a[j] - c[j] - lam;
        long id = ((long)kz * ny + j) * nkx + kx;
        xr[j] = spec[2 * id];
        xi[j] = spec[2 * id + 1];
      }
      int singular = (kx == 0 && kz == 0);
      if (singular) { b[0] = 1.0; c[0] = 0.0; xr[0] = 0.0; xi[0] = 0.0; }
      thomas(ny, a, b, c, xr, cw);
      thomas(ny, a, b, c, xi, cw);
      if (singular) {
        double mr = 0.0, mi = 0.0;
        if (g->yf) {   /* volume-weighted mean */
          for (int j = 0; j < ny; ++j) { mr += xr[j] * dyc(g, j); mi += xi[j] * dyc(g, j); }
          mr /= g->yf[ny]; mi /= g->yf[ny];
        } else {
          for (int j = 0; j < ny; ++j) { mr += xr[j]; mi += xi[j]; }
          mr /= ny; mi /= ny;
        }
        for (int j = 0; j < ny; ++j) { xr[j] -= mr; xi[j] -= mi; }
      }
      for (int j = 0; j < ny; ++j) {
        long id = ((long)kz * ny + j) * nkx + kx;
        spec[2 * id] = xr[j];
        spec[2 * id + 1] = xi[j];
      }
    }
    free(a);
  }
}

/* L_c = D G on the pressure grid with homogeneous Neumann walls (Eq. elliptic). */
void orc_lap_c(const orc_grid* g, const double* phi, double* out) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        double c0 = phi[cidx(g, i, j, k)];
        double lx = (phi[cidx(g, wrap(i + 1, nx), j, k)] - 2.0 * c0 + phi[cidx(g, wrap(i - 1, nx), j, k)]) /
                    (g->dx * g->dx);
        double lz = (phi[cidx(g, i, j, wrap(k + 1, nz))] - 2.0 * c0 + phi[cidx(g, i, j, wrap(k - 1, nz))]) /
                    (g->dz * g->dz);
        double up = (j + 1 < ny) ? (phi[cidx(g, i, j + 1, k)] - c0) : 0.0;
        double dn = (j > 0) ? (c0 - phi[cidx(g, i, j - 1, k)]) : 0.0;
        double ly = g->yf ? (up / dyf(g, j + 1) - dn / dyf(g, j)) / dyc(g, j) : (up - dn) / (g->dy * g->dy);
        out[cidx(g, i, j, k)] = lx + ly + lz;
      }
}

/* Projection (Eq. projection) and pressure update (Eq. update_pressure):
 *   u^{s+1} = uhat - alpha dt G phi   (v on the wall planes untouched)
 *   p^{s+1} = p^s + phi - alpha dt / (2 Re) L_c phi.
 * lapphi is L_c phi from orc_lap_c. */
void orc_project(const orc_grid* g, double* u, double* v, double* w, double* p, const double* phi,
                 const double* lapphi, double adt, double re) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        double c0 = phi[cidx(g, i, j, k)];
        u[fidx(g, 0, i, j, k)] -= adt * (c0 - phi[cidx(g, wrap(i - 1, nx), j, k)]) / g->dx;
        w[fidx(g, 2, i, j, k)] -= adt * (c0 - phi[cidx(g, i, j, wrap(k - 1, nz))]) / g->dz;
        if (j >= 1) v[fidx(g, 1, i, j, k)] -= adt * (c0 - phi[cidx(g, i, j - 1, k)]) / dyf(g, j);
        p[cidx(g, i, j, k)] += c0 - adt / (2.0 * re) * lapphi[cidx(g, i, j, k)];
      }
}

/* ------------------------------------------------------------------ */
/* Hydrodynamic loads on the surface (Section 3.3) and the pressure of  */
/* the boundary cells (Section 3.2, post-processing).                   */
/*                                                                      */
/* Markers are the triangle centroids X^l with the oriented unit normal */
/* n^l and area A^l.  A probe x^e = X^l + h n^l (h the IB probe length, */
/* twice the cell diagonal) is cast into the fluid; p and the velocity  */
/* gradient there come from second-order moving-least-squares fits and  */
/* are carried back to the wall by the Taylor series of the paper:      */
/*   p^l = p^e - h dp/dn + h^2/2 d2p/dn2,                               */
/*   grad u^l = grad u^e - h d(grad u)/dn  (a quadratic fit has no      */
/*   third derivatives, so the h^2 term of grad u vanishes);            */
/*   t^l = -p^l n + (grad u^l + grad u^l^T) n / Re,                     */
/*   F = sum t^l A^l,  M = sum (X^l - X^p) x t^l A^l.                   */
/* Readings (the MLS kernel is defined in a cited work, not here): the  */
/* fit of each quantity uses the 4 x 4 x 4 nearest nodes of its own     */
/* lattice around x^e (indices wrap in x and z, are clamped to the      */
/* stored planes in y), Gaussian weights exp(-(r/diag)^2), the basis    */
/* 1, xi, xi^2 and cross terms in xi = (x - x^e)/diag; nodes on the     */
/* other side of the marker's plane ((x - X^l).n <= 0) and, for p,      */
/* boundary cells are left out; with fewer than 10 weighted nodes the   */
/* fit drops to linear.  sides = 2 adds the loads of the opposite face  */
/* (normal -n) of the same triangle, for zero-thickness surfaces.       */
/* ------------------------------------------------------------------ */
static void node_xyz4(const orc_grid* g, int lat, long i, long j, long k, double x[3]) {
  /* lat 0..2: the u, v, w lattices; 3: cell centres */
  double off[3] = {0.5, 0.5, 0.5};
  if (lat < 3) off[lat] = 0.0;
  x[0] = ((double)i + off[0]) * g->dx;
  x[1] = ((double)j + off[1]) * g->dy;
  x[2] = ((double)k + off[2]) * g->dz;
}

/* Cholesky solve of the m x m SPD system M c = b (in place); 0 if not SPD */
static int chol_solve(int m, double* M, double* b) {
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = M[i * m + j];
      for (int k = 0; k < j; ++k) s -= M[i * m + k] * M[j * m + k];
      if (i == j) {
        if (!(s > 0.0)) return 0;
        M[i * m + i] = sqrt(s);
      } else {
        M[i * m + j] = s / M[j * m + j];
      }
    }
  }
  for (int i = 0; i < m; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= M[i * m + k] * b[k];
    b[i] = s / M[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < m; ++k) s -= M[k * m + i] * b[k];
    b[i] = s / M[i * m + i];
  }
  return 1;
}

/* Quadratic MLS fit of quantity f on lattice `lat` around xe; returns the
 * value, gradient and Hessian there.  Side test against (X, n); skip[]
 * (optional, per cell) excludes boundary cells. */
static void mls_fit(const orc_grid* g, int lat, const double* f, const uint8_t* skip, const double xe[3],
                    const double X[3], const double n[3], double* val, double grad[3], double H[9]) {
  const double del[3] = {g->dx, g->dy, g->dz};
  const double diag = sqrt(diag2_of(g));
  double off[3] = {0.5, 0.5, 0.5};
  if (lat < 3) off[lat] = 0.0;
  long planes = lat == 1 ? g->ny + 1 : g->ny;
  long i0[3];
  for (int d = 0; d < 3; ++d) i0[d] = (long)floor(xe[d] / del[d] - off[d]) - 1;
  if (i0[1] < 0) i0[1] = 0;
  if (i0[1] > planes - 4) i0[1] = planes - 4;
  double M[100] = {0}, b[10] = {0};
  int used = 0;
  for (int a = 0; a < 4; ++a)
    for (int bb = 0; bb < 4; ++bb)
      for (int c = 0; c < 4; ++c) {
        long ii = i0[0] + a, jj = i0[1] + bb, kk = i0[2] + c;
        double x[3];
        node_xyz4(g, lat, ii, jj, kk, x);
        double side = (x[0] - X[0]) * n[0] + (x[1] - X[1]) * n[1] + (x[2] - X[2]) * n[2];
        if (!(side > 0.0)) continue;
        long iw = wrap(ii, g->nx), kw = wrap(kk, g->nz);
        long id = (kw * planes + jj) * g->nx + iw;
        if (skip && skip[id]) continue;
        double xi[3], r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          xi[d] = (x[d] - xe[d]) / diag;
          r2 += xi[d] * xi[d];
        }
        double w = exp(-r2);
        double P[10] = {1.0, xi[0], xi[1], xi[2], xi[0] * xi[0], xi[1] * xi[1], xi[2] * xi[2],
                        xi[0] * xi[1], xi[0] * xi[2], xi[1] * xi[2]};
        for (int r = 0; r < 10; ++r) {
          b[r] += w * P[r] * f[id];
          for (int s = 0; s < 10; ++s) M[r * 10 + s] += w * P[r] * P[s];
        }
        ++used;
      }
  double cfs[10] = {0};
  int ok = 0;
  if (used >= 10) {
    double Mc[100], bc[10];
    memcpy(Mc, M, sizeof(Mc));
    memcpy(bc, b, sizeof(bc));
    if (chol_solve(10, Mc, bc)) {
      memcpy(cfs, bc, sizeof(bc));
      ok = 1;
    }
  }
  if (!ok) { /* linear fit: the leading 4 x 4 block */
    double Ml[16], bl[4];
    for (int r = 0; r < 4; ++r) {
      bl[r] = b[r];
      for (int s = 0; s < 4; ++s) Ml[r * 4 + s] = M[r * 10 + s];
    }
    if (chol_solve(4, Ml, bl))
      for (int r = 0; r < 4; ++r) cfs[r] = bl[r];
  }
  *val = cfs[0];
  for (int d = 0; d < 3; ++d) grad[d] = cfs[1 + d] / diag;
  const double id2 = 1.0 / (diag * diag);
  H[0] = 2.0 * cfs[4] * id2; H[4] = 2.0 * cfs[5] * id2; H[8] = 2.0 * cfs[6] * id2;
  H[1] = H[3] = cfs[7] * id2; H[2] = H[6] = cfs[8] * id2; H[5] = H[7] = cfs[9] * id2;
}

/* Traction at one marker and side: probe, fits, Taylor series. */
static void marker_traction(const orc_grid* g, const double* u, const double* v, const double* w, const double* p,
                            const uint8_t* isb, double re, const double X[3], const double n[3], double t[3],
                            double* pwall) {
  const double h = 2.0 * sqrt(diag2_of(g));
  double xe[3];
  for (int d = 0; d < 3; ++d) xe[d] = X[d] + h * n[d];
  double pe, gp[3], Hp[9];
  mls_fit(g, 3, p, isb, xe, X, n, &pe, gp, Hp);
  const double dpn = gp[0] * n[0] + gp[1] * n[1] + gp[2] * n[2];
  double d2pn = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) d2pn += n[a] * Hp[a * 3 + b] * n[b];
  const double pl = pe - h * dpn + 0.5 * h * h * d2pn;
  double G[9];   /* G[i*3 + j] = d u_i / d x_j at the wall */
  const double* comp[3] = {u, v, w};
  for (int i = 0; i < 3; ++i) {
    double val, gr[3], H[9];
    mls_fit(g, i, comp[i], NULL, xe, X, n, &val, gr, H);
    for (int j = 0; j < 3; ++j) {
      double Hn = H[j * 3 + 0] * n[0] + H[j * 3 + 1] * n[1] + H[j * 3 + 2] * n[2];
      G[i * 3 + j] = gr[j] - h * Hn;
    }
  }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += (G[i * 3 + j] + G[j * 3 + i]) * n[j];
    t[i] = -pl * n[i] + s / re;
  }
  *pwall = pl;
}

/* Loads of all triangles: tr[6 nt] = per triangle the force t A and the
 * torque (X - pole) x t A (summed over the sides), pwall[nt] the wall
 * pressure p^l on the normal's side; F, M the sums in triangle order. */
void orc_loads(const orc_grid* g, const double* xyz, int ntri, const int* tri, const double* u, const double* v,
               const double* w, const double* p, const uint8_t* isb, double re, int sides, const double* pole,
               double* tr, double* pwall, double* F, double* M) {
  for (int d = 0; d < 3; ++d) F[d] = M[d] = 0.0;
  for (long t = 0; t < ntri; ++t) {
    const double *a, *b, *c;
    tri_vertices(xyz, tri, t, &a, &b, &c);
    double X[3], e1[3], e2[3], nn[3];
    for (int d = 0; d < 3; ++d) {
      X[d] = (a[d] + b[d] + c[d]) / 3.0;
      e1[d] = b[d] - a[d];
      e2[d] = c[d] - a[d];
    }
    nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    const double area = 0.5 * len;
    double ft[3] = {0, 0, 0};
    for (int sd = 0; sd < sides; ++sd) {
      double n[3], tt[3], pw;
      for (int d = 0; d < 3; ++d) n[d] = (sd == 0 ? 1.0 : -1.0) * nn[d] / len;
      marker_traction(g, u, v, w, p, isb, re, X, n, tt, &pw);
      if (sd == 0) pwall[t] = pw;
      for (int d = 0; d < 3; ++d) ft[d] += tt[d] * area;
    }
    double r[3] = {X[0] - pole[0], X[1] - pole[1], X[2] - pole[2]};
    double m[3] = {r[1] * ft[2] - r[2] * ft[1], r[2] * ft[0] - r[0] * ft[2], r[0] * ft[1] - r[1] * ft[0]};
    for (int d = 0; d < 3; ++d) {
      tr[6 * t + d] = ft[d];
      tr[6 * t + 3 + d] = m[d];
      F[d] += ft[d];
      M[d] += m[d];
    }
  }
}

/* Pressure of the boundary cells (Section 3.2): not defined by the
 * solution there; the value at the probe point x^e = X + h N/|N| of the
 * cell centre (X its closest point on the owning triangle of the cell's
 * lower u face), trilinear from the surrounding cell centres (zero normal
 * gradient at the wall).  q[] = p with the boundary cells replaced. */
void orc_pressure_recon(const orc_grid* g, const double* p, const uint8_t* isb, const int32_t* own_u,
                        const double* xyz, const int* tri, double* q) {
  const long nx = g->nx, ny = g->ny, nz = g->nz, n = nx * ny * nz;
  const double h = 2.0 * sqrt(diag2_of(g));
  for (long id = 0; id < n; ++id) q[id] = p[id];
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        const long id = (k * ny + j) * nx + i;
        if (!isb[id]) continue;
        const int32_t t = own_u[id];   /* u grid and cells share the [k][j][i] layout */
        if (t < 0) continue;
        const double *a, *b, *c3;
        tri_vertices(xyz, tri, t, &a, &b, &c3);
        double x[3], X[3], wb[3], N[3];
        node_xyz4(g, 3, i, j, k, x);
        /* the periodic image of the centre nearest to the triangle */
        const double cx = (a[0] + b[0] + c3[0]) / 3.0, cz = (a[2] + b[2] + c3[2]) / 3.0;
        x[0] += g->lx * round((cx - x[0]) / g->lx);
        x[2] += g->lz * round((cz - x[2]) / g->lz);
        orc_closest_point(x, a, b, c3, X, wb);
        double nl = 0.0;
        for (int d = 0; d < 3; ++d) {
          N[d] = x[d] - X[d];
          nl += N[d] * N[d];
        }
        nl = sqrt(nl);
        if (nl == 0.0) {   /* centre on the surface: the triangle's normal */
          double e1[3], e2[3];
          for (int d = 0; d < 3; ++d) { e1[d] = b[d] - a[d]; e2[d] = c3[d] - a[d]; }
          N[0] = e1[1] * e2[2] - e1[2] * e2[1];
          N[1] = e1[2] * e2[0] - e1[0] * e2[2];
          N[2] = e1[0] * e2[1] - e1[1] * e2[0];
          nl = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        }
        double xe[3], pe;
        for (int d = 0; d < 3; ++d) xe[d] = X[d] + h * N[d] / nl;
        if (trilinear(g, 3, p, xe, &pe) == 0) q[id] = pe;
      }
}
