/*
 * Seeded synthetic inputs for the FTLE path: node coordinates and CSR
 * neighbour lists of structured-topology meshes.
 *
 * This module holds none of the FTLE arithmetic. It only builds what the
 * method takes as input: points, and each point's precomputed list of mesh
 * neighbours (the host-side neighbour precomputation of the paper's
 * "decoupled" design, Section 2.2).  Both the CUDA path and the FP64 oracle
 * read its output; neither is linked into it.
 *
 * Meshes are n[0] x n[1] (x n[2]) lattices over an axis-aligned box, nodes in
 * lexicographic order (x fastest), spacing h_d = (hi_d - lo_d) / (n_d - 1).
 * Stencils (neighbour offsets in lattice units, kept only when in bounds):
 *   FTLEIN_AXIS : +-e_d                    (4 in 2D, 6 in 3D; the paper's list)
 *   FTLEIN_TRI  : +-e_x, +-e_y, +-(e_x+e_y) (2D, each cell split along the
 *                 (i,j)-(i+1,j+1) diagonal: the mesh edges of the triangulation)
 *   FTLEIN_KUHN : +-e_x,+-e_y,+-e_z, +-(e_x+e_y), +-(e_x+e_z), +-(e_y+e_z),
 *                 +-(e_x+e_y+e_z) (3D, each hex split into the 6 Kuhn tetrahedra
 *                 around its main diagonal: the edges of that tetrahedralisation)
 * Each CSR row lists its neighbours in ascending index order; the adjacency is
 * symmetric and never contains the node itself.
 *
 * Jitter: node coordinate d moves by (2u - 1) * jitter * h_d, u in [0,1) from
 * SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based stream:
 * draw number k of seed s is mix64(s + (k + 1) * 0x9E3779B97F4A7C15), with
 * k = node_index * dim + d, and u = (r >> 11) * 2^-53.  Nodes on a face of the
 * box keep the coordinate normal to that face (so corners do not move), but
 * still consume their draws so every node's jitter depends only on its index.
 */
#include <stdint.h>
#include <stddef.h>

#define FTLEIN_AXIS 0
#define FTLEIN_TRI 1
#define FTLEIN_KUHN 2

static uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Uniform double in [0, 1) from draw k of the stream `seed`. */
double ftlein_uniform(uint64_t seed, uint64_t k) {
  return (double)(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

/* Raw 64-bit draw k of the stream `seed`. */
uint64_t ftlein_draw(uint64_t seed, uint64_t k) { return splitmix64_at(seed, k); }

/* Fill `out` (SoA [dim][N], N = prod n) with jittered lattice coordinates in
 * double precision.  Returns 0, or -1 on bad arguments. */
int ftlein_coords(int dim, const int64_t* n, const double* lo, const double* hi,
                  double jitter, uint64_t seed, double* out) {
  if (dim < 2 || dim > 3 || !n || !lo || !hi || !out) return -1;
  int64_t N = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 2) return -1;
    N *= n[d];
  }
  double h[3];
  for (int d = 0; d < dim; ++d) h[d] = (hi[d] - lo[d]) / (double)(n[d] - 1);
  for (int64_t i = 0; i < N; ++i) {
    int64_t rem = i, idx[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      idx[d] = rem % n[d];
      rem /= n[d];
    }
    for (int d = 0; d < dim; ++d) {
      double base = (idx[d] == n[d] - 1) ? hi[d] : lo[d] + (double)idx[d] * h[d];
      double u = ftlein_uniform(seed, (uint64_t)i * (uint64_t)dim + (uint64_t)d);
      int on_face = (idx[d] == 0) || (idx[d] == n[d] - 1);
      out[(int64_t)d * N + i] = on_face ? base : base + (2.0 * u - 1.0) * jitter * h[d];
    }
  }
  return 0;
}

static int stencil_offsets(int dim, int stencil, int off[][3]) {
  int m = 0;
  if (dim == 2 && stencil == FTLEIN_AXIS) {
    int o[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    for (int k = 0; k < 4; ++k) { off[m][0] = o[k][0]; off[m][1] = o[k][1]; off[m][2] = 0; ++m; }
  } else if (dim == 2 && stencil == FTLEIN_TRI) {
    int o[6][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}};
    for (int k = 0; k < 6; ++k) { off[m][0] = o[k][0]; off[m][1] = o[k][1]; off[m][2] = 0; ++m; }
  } else if (dim == 3 && stencil == FTLEIN_AXIS) {
    for (int d = 0; d < 3; ++d)
      for (int s = -1; s <= 1; s += 2) { off[m][0] = off[m][1] = off[m][2] = 0; off[m][d] = s; ++m; }
  } else if (dim == 3 && stencil == FTLEIN_KUHN) {
    /* the seven edge directions of a Kuhn tetrahedron path 0 -> e_a -> e_a+e_b -> (1,1,1) */
    int o[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
    for (int k = 0; k < 7; ++k)
      for (int s = -1; s <= 1; s += 2) {
        off[m][0] = s * o[k][0]; off[m][1] = s * o[k][1]; off[m][2] = s * o[k][2]; ++m;
      }
  } else {
    return -1;
  }
  return m;
}

/* Offsets sorted by the linear index they map to, so each row comes out ascending. */
static void sort_offsets(int m, int off[][3], const int64_t* n, int dim) {
  for (int a = 1; a < m; ++a)
    for (int b = a; b > 0; --b) {
      int64_t la = off[b][0] + (dim > 1 ? off[b][1] * n[0] : 0) + (dim > 2 ? off[b][2] * n[0] * n[1] : 0);
      int64_t lb = off[b - 1][0] + (dim > 1 ? off[b - 1][1] * n[0] : 0) +
                   (dim > 2 ? off[b - 1][2] * n[0] * n[1] : 0);
      if (la < lb) {
        for (int c = 0; c < 3; ++c) { int t = off[b][c]; off[b][c] = off[b - 1][c]; off[b - 1][c] = t; }
      } else {
        break;
      }
    }
}

/* Number of stored neighbours; -1 on bad arguments or when it exceeds int32. */
int64_t ftlein_nnz(int dim, const int64_t* n, int stencil) {
  int off[16][3];
  int m = stencil_offsets(dim, stencil, off);
  if (m < 0) return -1;
  int64_t nnz = 0;
  for (int k = 0; k < m; ++k) {
    int64_t cnt = 1;
    for (int d = 0; d < dim; ++d) {
      int64_t a = off[k][d] < 0 ? -off[k][d] : off[k][d];
      cnt *= (n[d] > a) ? (n[d] - a) : 0;
    }
    nnz += cnt;
  }
  if (nnz > 2147483647LL) return -1;
  return nnz;
}

/* Fill row_ptr[N+1] and col_idx[nnz] (int32).  Returns nnz or -1. */
int64_t ftlein_csr(int dim, const int64_t* n, int stencil, int32_t* row_ptr, int32_t* col_idx) {
  int off[16][3];
  int m = stencil_offsets(dim, stencil, off);
  if (m < 0 || !row_ptr || !col_idx) return -1;
  int64_t nnz_expect = ftlein_nnz(dim, n, stencil);
  if (nnz_expect < 0) return -1;
  sort_offsets(m, off, n, dim);
  int64_t N = 1;
  for (int d = 0; d < dim; ++d) N *= n[d];
  if (N > 2147483647LL) return -1;
  int64_t nz = 0;
  for (int64_t i = 0; i < N; ++i) {
    int64_t rem = i, idx[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) { idx[d] = rem % n[d]; rem /= n[d]; }
    row_ptr[i] = (int32_t)nz;
    for (int k = 0; k < m; ++k) {
      int ok = 1;
      int64_t j = 0, stride = 1;
      for (int d = 0; d < dim; ++d) {
        int64_t c = idx[d] + off[k][d];
        if (c < 0 || c >= n[d]) { ok = 0; break; }
        j += c * stride;
        stride *= n[d];
      }
      if (ok) col_idx[nz++] = (int32_t)j;
    }
  }
  row_ptr[N] = (int32_t)nz;
  return nz == nnz_expect ? nz : -1;
}
