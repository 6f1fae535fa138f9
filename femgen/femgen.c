/*
 * femgen.c -- seeded synthetic input generator for the sparse SPD systems
 * that the solver is exercised on.
 *
 * The paper's own matrix (a 30 880 x 30 880 stiffness matrix from an
 * electrical-machine finite-element model, Section III) is not available, so
 * this module produces stand-ins of the same kind: the stiffness matrix of
 * linear (P1) tetrahedral finite elements for -div(c grad u) on a jittered
 * structured node grid, each grid cube cut into the 6 Kuhn tetrahedra that
 * share the cube's main diagonal, with a piecewise-constant coefficient c
 * (1 in the background, `contrast` inside seeded boxes, standing in for
 * iron/air) and the Dirichlet nodes of all six faces eliminated.
 *
 * This file is INPUT PRODUCTION ONLY.  It holds no conjugate-gradient or
 * sparse matrix-vector arithmetic: the right-hand side b = A x* is assembled
 * element by element (b_i = sum over the tetrahedra that touch node i of the
 * element matrix row times x* on that element), never by multiplying the
 * assembled sparse matrix.  Both the CPU oracle and the GPU library consume
 * what it writes; it depends on neither.
 *
 * Determinism: every random number is a pure function of (seed, counter)
 * through the SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), so the output does not
 * depend on the thread count.  Rows are assembled independently ("row
 * centric"): row i sums the element contributions of the tetrahedra that
 * contain node i in increasing (cube, tetrahedron) order, so A_ij and A_ji
 * are sums of the same bitwise-identical terms in the same order and the
 * assembled matrix is exactly symmetric.  Build with -ffp-contract=off so
 * that x86 and Arm hosts produce identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FG_MAX_INCL 16

typedef struct {
  int32_t nx, ny, nz;     /* node grid, including the boundary nodes */
  int32_t n_incl;         /* number of box-shaped inclusions (<= 16) */
  int32_t dirichlet;      /* 1: drop all boundary nodes; 0: keep every node */
  int32_t pad_;
  double jitter;          /* interior-node jitter amplitude, in units of h */
  double contrast;        /* coefficient inside the inclusions (1 outside) */
  uint64_t seed_mesh;     /* jitter and inclusion boxes */
  uint64_t seed_x;        /* manufactured solution x* ~ U(-1, 1) */
} femgen_params;

/* ---------------------------------------------------------------- RNG --- */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
/* uniform double in [0, 1) from (seed, counter) */
static double fg_uniform(uint64_t seed, uint64_t ctr) {
  uint64_t h = splitmix64(splitmix64(seed) ^ (ctr * 0xD1342543DE82EF95ull + 0x632BE59BD9B4E019ull));
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}
double femgen_uniform(uint64_t seed, uint64_t ctr) { return fg_uniform(seed, ctr); }

/* ------------------------------------------------------------ geometry --- */
/* The 15 node offsets of the Kuhn pattern, sorted by their effect on the
 * lexicographic (k, j, i) node order so that a row's columns come out sorted. */
static const int OFF[15][3] = {
    {-1, -1, -1}, {0, -1, -1}, {-1, 0, -1}, {0, 0, -1}, {-1, -1, 0},
    {0, -1, 0},   {-1, 0, 0},  {0, 0, 0},   {1, 0, 0},  {0, 1, 0},
    {1, 1, 0},    {0, 0, 1},   {1, 0, 1},   {0, 1, 1},  {1, 1, 1}};
/* code of offset (di,dj,dk) = CODE[(dk+1)*9 + (dj+1)*3 + (di+1)], -1 if not a pattern offset */
static int CODE[27];
/* Kuhn tetrahedra: 4 corners each, as bit masks (bit0 = +x, bit1 = +y, bit2 = +z) */
static int TET[6][4];
static int tables_ready = 0;

static void fg_tables(void) {
  if (tables_ready) return;
  for (int c = 0; c < 27; ++c) CODE[c] = -1;
  for (int c = 0; c < 15; ++c) CODE[(OFF[c][2] + 1) * 9 + (OFF[c][1] + 1) * 3 + (OFF[c][0] + 1)] = c;
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int t = 0; t < 6; ++t) {
    int v1 = 1 << perm[t][0], v2 = v1 | (1 << perm[t][1]);
    /* orientation of the undistorted tetrahedron (0, v1, v2, 7) equals the
     * permutation parity; odd permutations get v1 and v2 swapped */
    int odd = (t == 1 || t == 2 || t == 5);
    TET[t][0] = 0;
    TET[t][1] = odd ? v2 : v1;
    TET[t][2] = odd ? v1 : v2;
    TET[t][3] = 7;
  }
  tables_ready = 1;
}

typedef struct {
  femgen_params p;
  double h;
  double box[FG_MAX_INCL][6]; /* lower corner (3), upper corner (3) */
  int32_t mx, my, mz;         /* unknown counts per axis */
  int32_t base;               /* 1 if boundary nodes are eliminated */
} fg_ctx;

static int fg_init(fg_ctx* c, const femgen_params* p) {
  fg_tables();
  if (p->nx < 2 || p->ny < 2 || p->nz < 2 || p->n_incl < 0 || p->n_incl > FG_MAX_INCL) return -1;
  c->p = *p;
  int mmax = p->nx > p->ny ? p->nx : p->ny;
  if (p->nz > mmax) mmax = p->nz;
  c->h = 1.0 / (double)(mmax - 1);
  for (int b = 0; b < p->n_incl; ++b) {
    for (int d = 0; d < 3; ++d) {
      /* counters above 2^62 keep the box draws apart from the node jitter draws */
      double lo = 0.6 * fg_uniform(p->seed_mesh, (1ull << 62) + 6ull * b + d);
      double ext = 0.2 + 0.2 * fg_uniform(p->seed_mesh, (1ull << 62) + 6ull * b + 3 + d);
      c->box[b][d] = lo;
      c->box[b][3 + d] = lo + ext;
    }
  }
  c->base = p->dirichlet ? 1 : 0;
  c->mx = p->nx - 2 * c->base;
  c->my = p->ny - 2 * c->base;
  c->mz = p->nz - 2 * c->base;
  if (c->mx < 1 || c->my < 1 || c->mz < 1) return -1;
  return 0;
}

static int is_boundary(const fg_ctx* c, int i, int j, int k) {
  return i == 0 || j == 0 || k == 0 || i == c->p.nx - 1 || j == c->p.ny - 1 || k == c->p.nz - 1;
}

/* unknown index of node (i,j,k), or -1 for an eliminated node */
static int64_t unk(const fg_ctx* c, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= c->p.nx || j >= c->p.ny || k >= c->p.nz) return -1;
  if (c->base && is_boundary(c, i, j, k)) return -1;
  return (int64_t)(i - c->base) + (int64_t)c->mx * ((int64_t)(j - c->base) + (int64_t)c->my * (k - c->base));
}

static void node_xyz(const fg_ctx* c, int i, int j, int k, double* x) {
  int ijk[3] = {i, j, k};
  uint64_t g = (uint64_t)i + (uint64_t)c->p.nx * ((uint64_t)j + (uint64_t)c->p.ny * (uint64_t)k);
  int bnd = is_boundary(c, i, j, k);
  for (int d = 0; d < 3; ++d) {
    x[d] = c->h * ijk[d];
    if (!bnd && c->p.jitter != 0.0)
      x[d] += c->p.jitter * c->h * (2.0 * fg_uniform(c->p.seed_mesh, 3ull * g + d) - 1.0);
  }
}

/* Element data of tetrahedron t of cube (ci,cj,ck): barycentric gradients
 * (rows of G), signed volume and coefficient.  Returns the volume. */
static double tet_element(const fg_ctx* c, int ci, int cj, int ck, int t, double G[4][3], double* coef) {
  double P[4][3];
  for (int v = 0; v < 4; ++v) {
    int m = TET[t][v];
    node_xyz(c, ci + (m & 1), cj + ((m >> 1) & 1), ck + ((m >> 2) & 1), P[v]);
  }
  double e1[3], e2[3], e3[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = P[1][d] - P[0][d];
    e2[d] = P[2][d] - P[0][d];
    e3[d] = P[3][d] - P[0][d];
  }
  double n1[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2], e2[0] * e3[1] - e2[1] * e3[0]};
  double n2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
  double n3[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double det = e1[0] * n1[0] + e1[1] * n1[1] + e1[2] * n1[2];
  for (int d = 0; d < 3; ++d) {
    G[1][d] = n1[d] / det;
    G[2][d] = n2[d] / det;
    G[3][d] = n3[d] / det;
    G[0][d] = -(G[1][d] + G[2][d] + G[3][d]);
  }
  double cen[3];
  for (int d = 0; d < 3; ++d) cen[d] = 0.25 * (P[0][d] + P[1][d] + P[2][d] + P[3][d]);
  double cc = 1.0;
  for (int b = 0; b < c->p.n_incl; ++b) {
    if (cen[0] >= c->box[b][0] && cen[0] <= c->box[b][3] && cen[1] >= c->box[b][1] &&
        cen[1] <= c->box[b][4] && cen[2] >= c->box[b][2] && cen[2] <= c->box[b][5]) {
      cc = c->p.contrast;
      break;
    }
  }
  *coef = cc;
  return det / 6.0;
}

static double kab(const double G[4][3], int a, int b, double cv) {
  return cv * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
}

/* --------------------------------------------------------------- API ---- */
/* Sizes of the system: n unknowns, nnz stored entries of the full matrix. */
int femgen_size(const femgen_params* p, int64_t* n, int64_t* nnz) {
  fg_ctx c;
  if (fg_init(&c, p)) return -1;
  int64_t cnt = 0;
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        if (unk(&c, i, j, k) < 0) continue;
        for (int o = 0; o < 15; ++o)
          if (unk(&c, i + OFF[o][0], j + OFF[o][1], k + OFF[o][2]) >= 0) ++cnt;
      }
  *n = (int64_t)c.mx * c.my * c.mz;
  *nnz = cnt;
  return 0;
}

/* Inclusion boxes as [lo_x, lo_y, lo_z, hi_x, hi_y, hi_z] per box. */
int femgen_boxes(const femgen_params* p, double* out) {
  fg_ctx c;
  if (fg_init(&c, p)) return -1;
  memcpy(out, c.box, sizeof(double) * 6 * p->n_incl);
  return 0;
}

/* Assemble the full CSR matrix (0-based, sorted columns), the manufactured
 * solution xstar (may be NULL -> not written, b then not written either) and
 * b = A xstar assembled element by element.  ptr has n+1 entries. */
int femgen_build(const femgen_params* p, int32_t* ptr, int32_t* idx, double* val, double* b, double* xstar) {
  fg_ctx c;
  if (fg_init(&c, p)) return -1;
  const int64_t n = (int64_t)c.mx * c.my * c.mz;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  /* pass 1: row lengths, in unknown order */
  int64_t run = 0;
  ptr[0] = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t r = unk(&c, i, j, k);
        if (r < 0) continue;
        for (int o = 0; o < 15; ++o)
          if (unk(&c, i + OFF[o][0], j + OFF[o][1], k + OFF[o][2]) >= 0) ++run;
        if (run > 0x7fffffffLL) return -2;
        ptr[r + 1] = (int32_t)run;
      }
  if (xstar)
    for (int64_t r = 0; r < n; ++r) xstar[r] = 2.0 * fg_uniform(p->seed_x, (uint64_t)r) - 1.0;
  /* pass 2: row-centric assembly; every row is independent */
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < nz; ++k) {
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t r = unk(&c, i, j, k);
        if (r < 0) continue;
        double acc[15];
        int valid[15];
        double brow = 0.0;
        for (int o = 0; o < 15; ++o) {
          acc[o] = 0.0;
          valid[o] = unk(&c, i + OFF[o][0], j + OFF[o][1], k + OFF[o][2]) >= 0;
        }
        /* cubes having (i,j,k) as a corner, in increasing cube index order */
        for (int dc = 1; dc >= 0; --dc)
          for (int db = 1; db >= 0; --db)
            for (int da = 1; da >= 0; --da) {
              int ci = i - da, cj = j - db, ck = k - dc;
              if (ci < 0 || cj < 0 || ck < 0 || ci > nx - 2 || cj > ny - 2 || ck > nz - 2) continue;
              int mine = da | (db << 1) | (dc << 2);
              for (int t = 0; t < 6; ++t) {
                int a = -1;
                for (int v = 0; v < 4; ++v)
                  if (TET[t][v] == mine) a = v;
                if (a < 0) continue;
                double G[4][3], coef;
                double vol = tet_element(&c, ci, cj, ck, t, G, &coef);
                double cv = coef * vol;
                for (int v = 0; v < 4; ++v) {
                  int m = TET[t][v];
                  int di = (m & 1) - da, dj = ((m >> 1) & 1) - db, dk = ((m >> 2) & 1) - dc;
                  int code = CODE[(dk + 1) * 9 + (dj + 1) * 3 + (di + 1)];
                  if (!valid[code]) continue; /* eliminated Dirichlet node */
                  double kv = kab(G, a, v, cv);
                  acc[code] += kv;
                  if (xstar) brow += kv * xstar[unk(&c, i + di, j + dj, k + dk)];
                }
              }
            }
        int64_t pos = ptr[r];
        for (int o = 0; o < 15; ++o) {
          if (!valid[o]) continue;
          idx[pos] = (int32_t)unk(&c, i + OFF[o][0], j + OFF[o][1], k + OFF[o][2]);
          val[pos] = acc[o];
          ++pos;
        }
        if (xstar && b) b[r] = brow;
      }
  }
  return 0;
}

/* Element data: for tetrahedron e = 6 * (ci + (nx-1) * (cj + (ny-1) * ck)) + t,
 * the unknown index of each of its 4 vertices (-1 for an eliminated node),
 * its unit-coefficient element matrix Kh = |V| G G' (4 x 4, row-major) and its
 * coefficient, so that A = sum_e coef_e Kh_e over the unknown vertices. */
int femgen_elements(const femgen_params* p, int32_t* nodes, double* kh, double* coef) {
  fg_ctx c;
  if (fg_init(&c, p)) return -1;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for schedule(static)
  for (int ck = 0; ck < nz - 1; ++ck)
    for (int cj = 0; cj < ny - 1; ++cj)
      for (int ci = 0; ci < nx - 1; ++ci)
        for (int t = 0; t < 6; ++t) {
          const int64_t e = 6 * ((int64_t)ci + (int64_t)(nx - 1) * ((int64_t)cj + (int64_t)(ny - 1) * ck)) + t;
          double G[4][3], cc;
          const double vol = tet_element(&c, ci, cj, ck, t, G, &cc);
          for (int v = 0; v < 4; ++v) {
            const int m = TET[t][v];
            nodes[4 * e + v] = (int32_t)unk(&c, ci + (m & 1), cj + ((m >> 1) & 1), ck + ((m >> 2) & 1));
            for (int w = 0; w < 4; ++w) kh[16 * e + 4 * v + w] = kab(G, v, w, vol);
          }
          coef[e] = cc;
        }
  return 0;
}

/* Smallest signed tetrahedron volume divided by h^3 (positive means every
 * element is positively oriented after jitter). */
double femgen_min_volume(const femgen_params* p) {
  fg_ctx c;
  if (fg_init(&c, p)) return -1.0;
  double vmin = 1e300;
  for (int k = 0; k < p->nz - 1; ++k)
    for (int j = 0; j < p->ny - 1; ++j)
      for (int i = 0; i < p->nx - 1; ++i)
        for (int t = 0; t < 6; ++t) {
          double G[4][3], coef;
          double v = tet_element(&c, i, j, k, t, G, &coef);
          if (v < vmin) vmin = v;
        }
  return vmin / (c.h * c.h * c.h);
}

/* Number of tetrahedra whose coefficient is the inclusion contrast. */
int64_t femgen_count_inclusion_tets(const femgen_params* p) {
  fg_ctx c;
  if (fg_init(&c, p)) return -1;
  int64_t cnt = 0;
  for (int k = 0; k < p->nz - 1; ++k)
    for (int j = 0; j < p->ny - 1; ++j)
      for (int i = 0; i < p->nx - 1; ++i)
        for (int t = 0; t < 6; ++t) {
          double G[4][3], coef;
          tet_element(&c, i, j, k, t, G, &coef);
          if (coef != 1.0) ++cnt;
        }
  return cnt;
}

/* Upper triangle (diagonal included) of a CSR matrix with sorted columns:
 * pure index selection.  uptr has n+1 entries; uidx/uval need room for the
 * kept entries (call with uidx == NULL to get only uptr). */
int femgen_upper(int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, int32_t* uptr,
                 int32_t* uidx, double* uval) {
  int64_t run = 0;
  uptr[0] = 0;
  for (int64_t r = 0; r < n; ++r) {
    for (int64_t q = ptr[r]; q < ptr[r + 1]; ++q) {
      if (idx[q] >= r) {
        if (uidx) {
          uidx[run] = idx[q];
          uval[run] = val[q];
        }
        ++run;
      }
    }
    uptr[r + 1] = (int32_t)run;
  }
  return 0;
}
