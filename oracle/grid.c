/*
 * Oracle (test infrastructure only): grids, cell walk and the non-local
 * core-skipping estimate, in FP64.
 *
 *   Sec. 3 (opening)       : per-cell density, temperature and velocity
 *   Sec. 2, Eq. tauH       : k_HI = n_HI sigma_0 (line-centre opacity per cm)
 *   Sec. 3.1.2             : cell-by-cell walk, x' = (x + k.u) sqrt(T/T') - k.u'
 *   Sec. 3.2.4, Eq. atauNL : a tau_NL = min over paths of sum a tau_0
 *
 * Geometry readings (the paper gives none):
 *   - cells are half-open [lo, hi); a point lying on a face belongs to the
 *     cell that its direction of travel enters (a zero direction component
 *     keeps the half-open rule);
 *   - after a crossing the exit coordinate is set exactly onto the face;
 *   - on exact ties between exit distances the lowest axis (x, y, z) wins;
 *   - periodic x/y (slab): leaving through an x or y face re-enters through
 *     the opposite face, the position shifted by the box length;
 *   - octree leaves are given as (level L, integer ijk at level L) inside the
 *     root box; a leaf spans lo + ijk s_L .. lo + (ijk+1) s_L, s_L = (hi-lo) 2^-L;
 *     crossing into an octree leaf locates the face point from the root.
 * Non-local estimate readings: paths run along the six coordinate axes from
 * the centre of each face of the cell outward (on octrees a centre lying on a
 * finer neighbour's split plane enters its upper side, the direction tie
 * rule for a zero direction component); the density reference is the
 * cell itself; a path continues while |n_i - n_ref| < f_NL n_ref and stops at
 * the domain edge (a periodic axis is followed for at most one period); the
 * path sum is sum a_i k_HI,i l_i with l_i the leaf length along the path.
 */
#include "grid.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

static void free_all(o_grid* g) {
  free(g->kHI); free(g->a); free(g->vth); free(g->u); free(g->kd); free(g->g);
  free(g->nHI); free(g->atau_nl); free(g->T); free(g->child); free(g->node_leaf);
  free(g->lev); free(g->ijk);
  memset(g, 0, sizeof(*g));
}

void o_grid_free(o_grid* g) { free_all(g); }

static int build_octree(const o_grid_in* in, o_grid* g) {
  int64_t n = in->n_leaves;
  g->lev = (uint8_t*)malloc((size_t)n);
  g->ijk = (uint32_t*)malloc((size_t)n * 3 * sizeof(uint32_t));
  if (!g->lev || !g->ijk) return -2;
  memcpy(g->lev, in->leaf_level, (size_t)n);
  memcpy(g->ijk, in->leaf_ijk, (size_t)n * 3 * sizeof(uint32_t));
  int64_t cap = 1024;
  g->child = (int64_t*)malloc((size_t)cap * 8 * sizeof(int64_t));
  g->node_leaf = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
  if (!g->child || !g->node_leaf) return -2;
  g->n_nodes = 1;
  for (int c = 0; c < 8; ++c) g->child[c] = -1;
  g->node_leaf[0] = -1;
  g->max_level = 0;
  for (int64_t l = 0; l < n; ++l) {
    int L = g->lev[l];
    if (L > 30) return -1;
    if (L > g->max_level) g->max_level = L;
    int64_t node = 0;
    for (int d = 0; d < L; ++d) {
      if (g->node_leaf[node] >= 0) return -1;            /* a leaf above this one */
      int shift = L - 1 - d;
      int cx = (g->ijk[3 * l + 0] >> shift) & 1;
      int cy = (g->ijk[3 * l + 1] >> shift) & 1;
      int cz = (g->ijk[3 * l + 2] >> shift) & 1;
      int ci = cx | (cy << 1) | (cz << 2);
      int64_t nx = g->child[8 * node + ci];
      if (nx < 0) {
        if (g->n_nodes == cap) {
          cap *= 2;
          int64_t* c2 = (int64_t*)realloc(g->child, (size_t)cap * 8 * sizeof(int64_t));
          int64_t* n2 = (int64_t*)realloc(g->node_leaf, (size_t)cap * sizeof(int64_t));
          if (!c2 || !n2) return -2;
          g->child = c2; g->node_leaf = n2;
        }
        nx = g->n_nodes++;
        for (int c = 0; c < 8; ++c) g->child[8 * nx + c] = -1;
        g->node_leaf[nx] = -1;
        g->child[8 * node + ci] = nx;
      }
      node = nx;
    }
    for (int c = 0; c < 8; ++c) if (g->child[8 * node + c] >= 0) return -1;  /* children below */
    if (g->node_leaf[node] >= 0) return -1;                                   /* duplicate */
    g->node_leaf[node] = l;
  }
  /* every internal node must have all 8 children (leaves tile the box) */
  for (int64_t v = 0; v < g->n_nodes; ++v) {
    if (g->node_leaf[v] >= 0) continue;
    for (int c = 0; c < 8; ++c) if (g->child[8 * v + c] < 0) return -1;
  }
  return 0;
}

int o_grid_build(const o_grid_in* in, o_grid* g) {
  memset(g, 0, sizeof(*g));
  g->kind = in->kind;
  g->periodic_xy = in->periodic_xy;
  for (int a = 0; a < 3; ++a) { g->lo[a] = in->lo[a]; g->hi[a] = in->hi[a]; }
  if (in->kind == 0) {
    g->n[0] = in->nx; g->n[1] = in->ny; g->n[2] = in->nz;
    if (g->n[0] <= 0 || g->n[1] <= 0 || g->n[2] <= 0) return -1;
    for (int a = 0; a < 3; ++a) g->h[a] = (g->hi[a] - g->lo[a]) / g->n[a];
    g->n_cells = (int64_t)g->n[0] * g->n[1] * g->n[2];
  } else if (in->kind == 1) {
    if (in->n_leaves <= 0 || in->periodic_xy) return -1;
    g->n_cells = in->n_leaves;
    int rc = build_octree(in, g);
    if (rc) { free_all(g); return rc; }
  } else {
    return -1;
  }
  int64_t n = g->n_cells;
  g->kHI = (double*)malloc((size_t)n * sizeof(double));
  g->a = (double*)malloc((size_t)n * sizeof(double));
  g->vth = (double*)malloc((size_t)n * sizeof(double));
  g->u = (double*)malloc((size_t)n * 3 * sizeof(double));
  g->kd = (double*)malloc((size_t)n * sizeof(double));
  g->g = (double*)malloc((size_t)n * sizeof(double));
  g->nHI = (double*)malloc((size_t)n * sizeof(double));
  g->atau_nl = (double*)calloc((size_t)n, sizeof(double));
  g->T = (double*)malloc((size_t)n * sizeof(double));
  if (!g->kHI || !g->a || !g->vth || !g->u || !g->kd || !g->g || !g->nHI || !g->atau_nl || !g->T) {
    free_all(g);
    return -2;
  }
  for (int64_t c = 0; c < n; ++c) {
    double T = in->T[c];
    if (!(T > 0.0) || !(in->n_HI[c] >= 0.0)) { free_all(g); return -1; }
    double vth = o_vth_kms(T);
    g->nHI[c] = in->n_HI[c];
    g->T[c] = T;
    g->kHI[c] = (double)in->n_HI[c] * o_sigma0(T);          /* Eq. tauH */
    g->a[c] = o_damping_a(T);
    g->vth[c] = vth;
    g->u[3 * c + 0] = (double)in->vx[c] / vth;              /* u = v / v_th */
    g->u[3 * c + 1] = (double)in->vy[c] / vth;
    g->u[3 * c + 2] = (double)in->vz[c] / vth;
    g->kd[c] = in->k_dust ? (double)in->k_dust[c] : 0.0;
    g->g[c] = o_recoil_g(T);
  }
  return 0;
}

/* Leaf/cell bounds. */
void o_cell_bounds(const o_grid* g, int64_t c, double clo[3], double chi[3]) {
  if (g->kind == 0) {
    int64_t i = c % g->n[0];
    int64_t j = (c / g->n[0]) % g->n[1];
    int64_t k = c / ((int64_t)g->n[0] * g->n[1]);
    int64_t id[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
      clo[a] = g->lo[a] + (double)id[a] * g->h[a];
      chi[a] = g->lo[a] + (double)(id[a] + 1) * g->h[a];
    }
  } else {
    int L = g->lev[c];
    for (int a = 0; a < 3; ++a) {
      double s = ldexp(g->hi[a] - g->lo[a], -L);
      clo[a] = g->lo[a] + (double)g->ijk[3 * c + a] * s;
      chi[a] = g->lo[a] + (double)(g->ijk[3 * c + a] + 1) * s;
    }
  }
}

/* Which side of a split plane the point goes to (half-open, direction rule). */
static int upper_side(double r, double split, double k) {
  if (r > split) return 1;
  if (r < split) return 0;
  return (k < 0.0) ? 0 : 1;
}

int64_t o_locate_cell(const o_grid* g, const double r[3], const double k[3]) {
  if (g->kind == 0) {
    int64_t id[3];
    for (int a = 0; a < 3; ++a) {
      double t = (r[a] - g->lo[a]) / g->h[a];
      double f = floor(t);
      int64_t i = (int64_t)f;
      if (t == f && k[a] < 0.0) i -= 1;
      if (i < 0 || i >= g->n[a]) return -1;
      id[a] = i;
    }
    return id[0] + (int64_t)g->n[0] * (id[1] + (int64_t)g->n[1] * id[2]);
  }
  /* octree: descend from the root */
  double blo[3], bhi[3];
  for (int a = 0; a < 3; ++a) {
    blo[a] = g->lo[a]; bhi[a] = g->hi[a];
    if (r[a] < blo[a] || r[a] > bhi[a]) return -1;
    if (r[a] == blo[a] && k[a] < 0.0) return -1;
    if (r[a] == bhi[a] && !(k[a] < 0.0)) return -1;
  }
  /* the split plane of a node at depth d is lo + (2i + 1) s_d (i: the node's
   * integer coordinate), the same number o_cell_bounds gives the leaf faces
   * lying in it, so a point snapped onto a face is classified exactly */
  int64_t node = 0;
  int depth = 0;
  int64_t ii[3] = {0, 0, 0};
  while (g->node_leaf[node] < 0) {
    int ci = 0;
    ++depth;
    for (int a = 0; a < 3; ++a) {
      double s = ldexp(g->hi[a] - g->lo[a], -depth);
      double mid = g->lo[a] + (double)(2 * ii[a] + 1) * s;
      int up = upper_side(r[a], mid, k[a]);
      ii[a] = 2 * ii[a] + up;
      ci |= up << a;
    }
    node = g->child[8 * node + ci];
  }
  return g->node_leaf[node];
}

int64_t o_octree_locate(const o_grid_in* gin, const double pos[3], const double dir[3]) {
  o_grid g;
  if (o_grid_build(gin, &g)) return -2;
  int64_t c = o_locate_cell(&g, pos, dir);
  o_grid_free(&g);
  return c;
}

/* Distance from r along k to the exit face of the cell [clo, chi); *axis gets
 * the exit axis (lowest on ties).  Negative distances are clamped to zero.  */
double o_exit_distance(const double clo[3], const double chi[3], const double r[3],
                       const double k[3], int* axis) {
  double best = INFINITY;
  int ax = -1;
  for (int a = 0; a < 3; ++a) {
    if (k[a] == 0.0) continue;
    double face = (k[a] > 0.0) ? chi[a] : clo[a];
    double d = (face - r[a]) / k[a];
    if (d < 0.0) d = 0.0;
    if (d < best) { best = d; ax = a; }
  }
  *axis = ax;
  return best;
}

/* After moving onto the exit face of cell c along axis ax, find the cell on
 * the other side.  r is updated in place (exit coordinate snapped onto the
 * face, periodic wrap applied).  Returns -1 when the packet leaves the box. */
int64_t o_next_cell(const o_grid* g, int64_t c, int ax, double r[3], const double k[3]) {
  double clo[3], chi[3];
  o_cell_bounds(g, c, clo, chi);
  r[ax] = (k[ax] > 0.0) ? chi[ax] : clo[ax];
  if (g->kind == 0) {
    int64_t id[3] = {c % g->n[0], (c / g->n[0]) % g->n[1], c / ((int64_t)g->n[0] * g->n[1])};
    id[ax] += (k[ax] > 0.0) ? 1 : -1;
    if (id[ax] < 0 || id[ax] >= g->n[ax]) {
      if (g->periodic_xy && ax < 2) {
        if (id[ax] < 0) { id[ax] = g->n[ax] - 1; r[ax] = g->hi[ax]; }
        else            { id[ax] = 0;            r[ax] = g->lo[ax]; }
      } else {
        return -1;
      }
    }
    return id[0] + (int64_t)g->n[0] * (id[1] + (int64_t)g->n[1] * id[2]);
  }
  return o_locate_cell(g, r, k);
}

/* Minimum distance from r to any face of cell c (Sec. 3.2.4, Eq. atau0min). */
double o_min_face_distance(const o_grid* g, int64_t c, const double r[3]) {
  double clo[3], chi[3];
  o_cell_bounds(g, c, clo, chi);
  double m = INFINITY;
  for (int a = 0; a < 3; ++a) {
    double d1 = r[a] - clo[a], d2 = chi[a] - r[a];
    if (d1 < m) m = d1;
    if (d2 < m) m = d2;
  }
  return m < 0.0 ? 0.0 : m;
}

/* Eq. atauNL for cells [c0, c1). */
static void atau_nl_range(o_grid* g, double f_nl, int64_t c0, int64_t c1) {
  for (int64_t c = c0; c < c1; ++c) {
    double nref = g->nHI[c];
    if (!(nref > 0.0) || !(f_nl > 0.0)) { g->atau_nl[c] = 0.0; continue; }
    double clo[3], chi[3];
    o_cell_bounds(g, c, clo, chi);
    double best = INFINITY;
    for (int dir = 0; dir < 6; ++dir) {
      int ax = dir >> 1;
      double k[3] = {0.0, 0.0, 0.0};
      k[ax] = (dir & 1) ? -1.0 : 1.0;
      double r[3];
      for (int a = 0; a < 3; ++a) {
        /* the centre of an octree leaf is the split plane of its level L + 1,
         * lo + (2i + 1) s_{L+1}, taken as that same number: where a finer
         * neighbour is split there, the path enters its upper side */
        if (g->kind == 1)
          r[a] = g->lo[a] + (double)(2 * (int64_t)g->ijk[3 * c + a] + 1) * ldexp(g->hi[a] - g->lo[a], -(g->lev[c] + 1));
        else
          r[a] = 0.5 * (clo[a] + chi[a]);
      }
      int64_t cur = c;
      double sum = 0.0;
      int64_t steps = 0;
      int64_t limit = (g->kind == 0) ? g->n[ax] - 1 : (int64_t)1 << 62;
      for (;;) {
        int64_t nx = o_next_cell(g, cur, ax, r, k);
        if (nx < 0 || nx == c) break;
        if (++steps > limit) break;
        double ni = g->nHI[nx];
        if (!(fabs(ni - nref) < f_nl * nref)) break;
        double blo[3], bhi[3];
        o_cell_bounds(g, nx, blo, bhi);
        sum += g->a[nx] * g->kHI[nx] * (bhi[ax] - blo[ax]);
        cur = nx;
      }
      if (sum < best) best = sum;
    }
    g->atau_nl[c] = best;
  }
}

typedef struct { o_grid* g; double f_nl; int64_t c0, c1; } nl_job;

static void* nl_worker(void* arg) {
  nl_job* j = (nl_job*)arg;
  atau_nl_range(j->g, j->f_nl, j->c0, j->c1);
  return NULL;
}

/* Eq. atauNL: cells are independent, so they are split across host threads. */
int o_atau_nl_grid(o_grid* g, double f_nl) {
  int nt = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nt < 1) nt = 1;
  if (nt > 64) nt = 64;
  if (g->n_cells < 4096) nt = 1;
  pthread_t th[64];
  nl_job jobs[64];
  int64_t per = (g->n_cells + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    jobs[t].g = g; jobs[t].f_nl = f_nl;
    jobs[t].c0 = t * per;
    jobs[t].c1 = (t + 1) * per < g->n_cells ? (t + 1) * per : g->n_cells;
    if (jobs[t].c0 > jobs[t].c1) jobs[t].c0 = jobs[t].c1;
    pthread_create(&th[t], NULL, nl_worker, &jobs[t]);
  }
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  return 0;
}

int o_atau_nl(const o_grid_in* gin, double f_nl, double* out) {
  o_grid g;
  int rc = o_grid_build(gin, &g);
  if (rc) return rc;
  o_atau_nl_grid(&g, f_nl);
  memcpy(out, g.atau_nl, (size_t)g.n_cells * sizeof(double));
  o_grid_free(&g);
  return 0;
}
