/* Oracle-internal grid representation (test infrastructure only). */
#ifndef COLT_ORACLE_GRID_H
#define COLT_ORACLE_GRID_H
#include "oracle.h"

typedef struct {
  int kind;
  int n[3];
  double lo[3], hi[3], h[3];
  int periodic_xy;
  int64_t n_cells;
  /* derived per-cell quantities, FP64 */
  double *kHI, *a, *vth, *u, *kd, *g, *nHI, *atau_nl, *T;
  /* octree */
  int64_t n_nodes;
  int max_level;
  int64_t* child;      /* 8 per node, -1 = none */
  int64_t* node_leaf;  /* leaf index or -1      */
  uint8_t* lev;
  uint32_t* ijk;
} o_grid;

int     o_grid_build(const o_grid_in* in, o_grid* g);
void    o_grid_free(o_grid* g);
void    o_cell_bounds(const o_grid* g, int64_t c, double clo[3], double chi[3]);
int64_t o_locate_cell(const o_grid* g, const double r[3], const double k[3]);
double  o_exit_distance(const double clo[3], const double chi[3], const double r[3],
                        const double k[3], int* axis);
int64_t o_next_cell(const o_grid* g, int64_t c, int ax, double r[3], const double k[3]);
double  o_min_face_distance(const o_grid* g, int64_t c, const double r[3]);
int     o_atau_nl_grid(o_grid* g, double f_nl);

#endif
