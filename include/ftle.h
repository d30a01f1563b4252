/*
 * ftle.h - C-ABI of libftle.so, the GB300 (sm_103a) FTLE hot path.
 *
 * What is computed (arXiv 2408.02758, "Finite-Time Lyapunov Exponent Calculation on FPGA using
 * High-Level Synthesis Tools"):
 *   - the flowmap phi_T(x0) of every mesh node, the input of the paper's FTLE kernel
 *     (Section 2.2: the flowmap and neighbour lists arrive precomputed), here integrated on the
 *     GPU by classic RK4 through an analytic velocity field;
 *   - the per-node FTLE core (Section 2.1, Table 1): least-squares flowmap gradient over the
 *     node's precomputed neighbour list (Section 2.2, "decoupled" algorithm),
 *     F = (sum_j dphi_j dx_j^T)(sum_j dx_j dx_j^T)^-1, dx_j = x_j - x_i, dphi_j = phi_j - phi_i,
 *     the Cauchy-Green tensor C = F^T F, its largest eigenvalue lambda_max, and
 *     FTLE = ln(sqrt(lambda_max)) / |T|.
 * The paper's neighbour list is a fixed-width list padded with -1 (Section 2.2); this library
 * takes the equivalent compressed form (CSR), where a short row simply has fewer entries.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller unless stated otherwise; the
 *     library never frees or retains them past the call.  Nothing persistent is allocated on
 *     the device (the batched plan holds a CUDA graph, see ftle_batch_plan_create).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue work and
 *     return after launch; results are ready when the stream reaches that point.
 *   - Return value: FTLE_OK (0) or a negative ftle_status.  Argument errors are detected on the
 *     host before anything is launched.  Conditions found on the device (degenerate
 *     neighbourhoods, nodes that took the FP64 path) are counted in the workspace header
 *     (ftle_counters), never by a trap.  ftle_last_error() gives a message for the last failing
 *     call of the calling thread.  No C++ exception crosses this boundary.
 *   - Thread-safe for calls on distinct streams with distinct output/workspace buffers.
 *   - Node coordinates are SoA: coords[d * n_nodes + i], d < dim.  Neighbour lists are CSR:
 *     the neighbours of node i are col_idx[row_ptr[i] .. row_ptr[i+1]), int32, 0 <= j < n_nodes.
 *     Kernels gather through these indices: ftle_validate_mesh checks them (the entry points do
 *     so themselves with ftle_options.validate_mesh = 1, ftle_compute_host always).
 *   - T < 0 integrates backward in time; |T| enters the FTLE formula.  The RK4 step is
 *     h = sign(T) |dt|, n = round(|T| / |dt|) steps from t0, stages at t_k, t_k + h/2 (twice),
 *     t_k + h with t_k = t0 + k h.
 */
#ifndef FTLE_H
#define FTLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FTLE_API_VERSION 1

typedef enum ftle_status {
  FTLE_OK = 0,
  FTLE_EINVAL = -1,        /* bad argument: null pointer, size, mode or flow/dimension mismatch */
  FTLE_ECUDA = -2,         /* a CUDA runtime call failed (message in ftle_last_error) */
  FTLE_EWORKSPACE = -3,    /* workspace missing or smaller than the *_workspace_bytes query */
  FTLE_EUNSUPPORTED = -4,  /* combination this build does not provide */
  FTLE_ERANGE = -5,        /* a size beyond a fixed limit (step count, nnz, static capacity) */
  FTLE_ENOMEM = -6         /* a host-side allocation failed (batch plans) */
} ftle_status;

/* Velocity fields u(x, t); parameters in ftle_flow.p:
 *   DOUBLE_GYRE (2D): p = {A, eps, omega}; f = a x^2 + b x, a = eps sin(omega t),
 *                     b = 1 - 2 eps sin(omega t); u = -pi A sin(pi f) cos(pi y),
 *                     v = pi A cos(pi f) sin(pi y) df/dx.
 *   ABC (3D):         p = {A, B, C}; u = A sin z + C cos y, v = B sin x + A cos z,
 *                     w = C sin y + B cos x.
 *   LINEAR (2D/3D):   u = M x, M row-major dim x dim in p[0 .. dim*dim).
 *   SADDLE (2D/3D):   u = (x, -y) in 2D, (x, -y, 0) in 3D. */
typedef enum ftle_flow_kind {
  FTLE_FLOW_DOUBLE_GYRE = 0,
  FTLE_FLOW_ABC = 1,
  FTLE_FLOW_LINEAR = 2,
  FTLE_FLOW_SADDLE = 3
} ftle_flow_kind;

/* Arithmetic of the path.
 *   FP64:  everything in double.  flowmap: double [dim][n]; ftle_out: double [n].
 *   FP32:  plain float RK4 and float gradient.  flowmap: float [dim][n]; ftle_out: float [n].
 *   FP32C: float RK4 stages with a compensated (two-sum) state and velocity evaluated at the
 *          compensated stage point; the flowmap is stored as (hi, lo) float pairs,
 *          flowmap: float2 [dim][n] (hi at even, lo at odd float index); gradient in float,
 *          with the FP64 path for the nodes where float cancels (see ftle_options.refine_kappa).
 *          ftle_out: float [n]. */
typedef enum ftle_precision { FTLE_PREC_FP64 = 0, FTLE_PREC_FP32 = 1, FTLE_PREC_FP32C = 2 } ftle_precision;

/* Neighbours implied by a structured lattice (ftle_mesh.stencil), offsets (ox, oy[, oz]):
 *   FTLE_STENCIL_AXIS: +-e_a on every axis (4 in 2D, 6 in 3D);
 *   FTLE_STENCIL_TRI (2D): +-e_x, +-e_y, +-(1, 1) (cells split along the (i,j)-(i+1,j+1) diagonal);
 *   FTLE_STENCIL_KUHN (3D): +-e_a, +-(e_x + e_y), +-(e_y + e_z), +-(e_x + e_z), +-(1, 1, 1) (cubes
 *   split into six tetrahedra around the main diagonal). */
typedef enum ftle_stencil {
  FTLE_STENCIL_NONE = 0,
  FTLE_STENCIL_AXIS = 1,
  FTLE_STENCIL_TRI = 2,
  FTLE_STENCIL_KUHN = 3
} ftle_stencil;

typedef struct ftle_mesh {
  int32_t dim;            /* 2 or 3 */
  int32_t coord_fp64;     /* 0: coords are float, 1: coords are double */
  int64_t n_nodes;        /* number of nodes, 0 <= n_nodes < 2^31 */
  int64_t nnz;            /* entries of col_idx (= row_ptr[n_nodes]), < 2^31 */
  const void* coords;     /* device, SoA [dim][n_nodes] */
  const int32_t* row_ptr; /* device [n_nodes + 1], non-decreasing, row_ptr[0] = 0 */
  const int32_t* col_idx; /* device [nnz] */
  /* Optional fixed-width form of the same lists, the paper's decoupled layout (Section 2.2):
   * ell_idx[s * n_nodes + i] is neighbour s of node i, -1 where a node has fewer than ell_width
   * neighbours.  When set (ell_width > 0, ell_idx != NULL) the float gradient kernel reads it
   * instead of the CSR rows (all slot loads independent and coalesced); the CSR arrays stay
   * required for the FP64 path, the refinement and the adjoint.  Build it with ftle_ell_from_csr. */
  int32_t ell_width;      /* 0: no fixed-width list */
  int32_t reserved;       /* must be 0 */
  const int32_t* ell_idx; /* device [ell_width][n_nodes] or NULL */
  /* Optional implicit neighbours of a structured lattice, the paper's regular access pattern
   * (Section 2.2) without any list: node i = ix + grid[0] (iy + grid[1] iz) has as neighbours
   * the stencil's offsets that stay inside the lattice, in ascending node order (the order of
   * sorted CSR rows).  When stencil != FTLE_STENCIL_NONE the float gradient kernel reads no
   * neighbour index (it takes precedence over ell_idx); the CSR arrays stay required for the FP64
   * path, the refinement and the adjoint, and must list the same neighbours (the float and FP64
   * paths would otherwise disagree).  grid[a] >= 2 on each axis, grid[2] = 1 in 2D, and
   * grid[0] grid[1] grid[2] = n_nodes; FTLE_EINVAL otherwise. */
  int32_t stencil;        /* ftle_stencil; 0: neighbours from the lists */
  int32_t grid[3];        /* lattice nodes per axis, x fastest */
} ftle_mesh;

typedef struct ftle_flow {
  int32_t kind;     /* ftle_flow_kind */
  int32_t reserved; /* must be 0 */
  double p[12];     /* parameters, layout per kind above */
} ftle_flow;

/* Device-side counters, at offset 0 of every workspace.  Read them with ftle_read_counters. */
typedef struct ftle_counters {
  unsigned long long n_flagged;    /* nodes whose gradient/eigenvalues went to the FP64 path */
  unsigned long long n_degenerate; /* nodes with a rank-deficient neighbourhood: FTLE = NaN */
  unsigned long long n_readvected; /* nodes re-advected in float-float by ftle_refine */
  unsigned long long reserved[4];
  unsigned long long n_wait_timeouts; /* bounded waits of a kernel that ran out (a stalled copy);
                                         the kernel's blocks stop, their outputs are incomplete */
} ftle_counters;

/* Optional tuning; pass NULL for defaults.  Zero fields mean "default". */
typedef struct ftle_options {
  double refine_kappa;    /* FP32/FP32C: node i takes the FP64 gradient (and, in ftle_refine,
                             the float-float re-advection) when ln(lambda_max) * h_i < refine_kappa,
                             h_i its RMS neighbour distance: the float flowmap's error relative to
                             h_i, divided by ln(lambda_max), bounds the FTLE's relative error.
                             Default 4e-4 when the field is 0; negative turns this test off (the
                             rank, conditioning and lambda_max - 1 < 0.01 checks remain). */
  int32_t advect_block;   /* threads per block of the advection kernel (multiple of 32) */
  int32_t advect_blocks_per_sm; /* blocks per SM the advection grid is sized for (default
                                   8192 / advect_block; a block loops over node tiles while
                                   the grid is smaller than the mesh) */
  int32_t grad_block;     /* threads per block of the gradient kernel (multiple of 32) */
  int32_t grad_tile;      /* nodes per gradient tile (multiple of grad_block) */
  int32_t refine_lanes;   /* re-advection: active lanes per 32-thread block (1..32); fewer lanes
                             spread a short node list over more SM sub-partitions (the 3D ABC
                             re-advection takes one warp per node and ignores it) */
  int32_t defer_fp64;     /* 1: ftle_gradient_eig leaves the flagged nodes' FP64 pass to the
                             ftle_refine that the caller runs next with these options, which
                             recomputes those nodes after the re-advection anyway (their outputs
                             stay NaN until then).  Ignored, and the pass runs, when ftle_refine
                             would not refine (FP32, or refine_kappa < 0).  ftle_compute does
                             this by itself. */
  int32_t validate_mesh;  /* 1: ftle_gradient_eig, ftle_compute and ftle_batch (and
                             ftle_batch_plan_create) first run ftle_validate_mesh on every mesh
                             they are given and return FTLE_EINVAL, with nothing else launched,
                             when an index is out of range.  The check synchronises the stream
                             once per mesh (it reads its counters back), so it is off by default;
                             ftle_compute_host always runs it. */
  int32_t grad_staging;   /* float gradient of compensated flowmaps: 0 brings each tile's
                             neighbour indices into shared memory by bulk copies (TMA) one tile
                             ahead of the computation (the fixed-width list: width 6 in 2D or 14
                             in 3D, n_nodes a multiple of 4, ell_idx 16-byte aligned; CSR rows:
                             col_idx 16-byte aligned), 1 reads the indices with plain loads.
                             Same results either way. */
  int32_t abc_refresh;    /* compensated ABC advection with the unchecked step (ftle_rotation_bounds
                             .unchecked): stage one's sines and cosines of the state are evaluated
                             afresh every abc_refresh steps and, in between, taken from the
                             previous step's stage four and turned by the rest of that step's
                             increment (a power of two in [1, 1024]; default 8; 1 evaluates them
                             at every step).  They are carried only while the step's angle bound
                             (ftle_rotation_bounds .angle_bound) stays within 0.032 rad; beyond
                             that every step evaluates them afresh whatever abc_refresh says. */
} ftle_options;

/* ---------------------------------------------------------------------------------- sizes */

/* Bytes of a flowmap buffer for `precision` (0 on bad arguments).  For FP32C the buffer holds the
 * (hi, lo) pairs float2 [dim][n] followed, at the next 256-byte boundary, by one 32-byte record
 * per node that the float gradient kernel reads (coordinates, hi parts and low parts packed:
 * 2D {x, y, hx, hy}{lx, ly, 0, 0}; 3D {x, y, z, hx}{hy, hz, lx, bf16(ly) | bf16(lz) << 16}).
 * A 2D FP32C flowmap then holds, each at the next 256-byte boundary, 7 more (hi, lo) states
 * float2 [2][n]: slot j is the state after min((j + 1) L, nsteps) steps, L = ceil(nsteps / 8),
 * the starting points from which ftle_refine re-advects 8 runs of a node side by side.
 * ftle_refine therefore takes the flowmap ftle_advect wrote with the same t0, T and dt. */
size_t ftle_flowmap_bytes(int32_t dim, int64_t n_nodes, int32_t precision);

/* Bytes of one checkpoint slot: the state alone (the FP32C (hi, lo) pairs, without records). */
size_t ftle_checkpoint_bytes(int32_t dim, int64_t n_nodes, int32_t precision);

/* Bytes of the workspace ftle_gradient_eig / ftle_refine / ftle_compute need for n_nodes:
 * counters header, the FP64-path node list and the re-advection mark set.  The workspace must
 * be 256-byte aligned.  Its contents need no initialisation; each call clears what it uses. */
size_t ftle_workspace_bytes(int64_t n_nodes);

/* --------------------------------------------------------------------------- single problem */

/* Flowmap by RK4 (the input of the FTLE core, Section 2.2).
 *   flowmap     device out, ftle_flowmap_bytes(dim, n, precision) bytes, layout per precision.
 *   checkpoints nullable device out: the state every ckpt_every steps for the adjoint
 *               (ftle_backward); ckpt_count = n_steps / ckpt_every + 1 slots of
 *               ftle_checkpoint_bytes each (slot s holds the state after s * ckpt_every steps).
 *   ckpt_every  > 0 when checkpoints is given, else ignored.
 * Errors: FTLE_EINVAL (null mesh/flow/flowmap, dt = 0, T = 0, flow kind not valid for dim,
 * coords precision not matching FP64 mode's need), FTLE_ERANGE (more than 2^31 - 1 steps). */
int ftle_advect(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt,
                int32_t precision, void* flowmap, void* checkpoints, int32_t ckpt_every,
                const ftle_options* opt, void* stream);

/* The bounds behind ftle_advect's unchecked steps (FTLE_PREC_FP32C, double gyre and ABC flow).
 * The compensated step evaluates stage one's sines and cosines and turns them for stages two to
 * four by the small stage angles (Taylor to third order), stage three from stage two's by the
 * angle differences to first order.  When the host bounds every angle and difference of a step
 * of size |dt| within the turns' limits, the kernels drop the per-step angle check (double gyre:
 * for nodes starting in its invariant domain [0, 2] x [0, 1]; ABC: everywhere):
 *   angle_bound  bound on every stage angle, radians (double gyre: the larger of pi f's and pi y's);
 *   diff_bound   bound on stage three's angle differences;
 *   angle_limit, diff_limit  the limits with their 1e-3 margin (0.05 and 3e-4 before it);
 *   unchecked    1 when both bounds are within their limits, else 0;
 *   carried      ABC: 1 when the unchecked step also carries stage one's sines and cosines from
 *                step to step (ftle_options.abc_refresh > 1 asks for it), i.e. unchecked and
 *                angle_bound within 0.032 rad (with the same margin); else 0.
 * Flows without the rotated step (linear, saddle): unchecked = 0, both bounds +inf.
 * Host only (no device work).  Errors: FTLE_EINVAL (null flow or out, unknown kind, parameters
 * or dt not finite, dt = 0). */
typedef struct {
  int32_t unchecked;
  int32_t carried;
  double angle_bound;
  double diff_bound;
  double angle_limit;
  double diff_limit;
} ftle_rotation_info;
int ftle_rotation_bounds(const ftle_flow* flow, double dt, ftle_rotation_info* out);

/* The FTLE core (Section 2.1, Table 1) over the CSR neighbour lists (Section 2.2).
 *   flowmap     device in (as written by ftle_advect for the same precision).
 *   ftle_out    device out [n_nodes]: float, or double for FTLE_PREC_FP64.  NaN where the
 *               neighbourhood is rank-deficient (fewer than dim neighbours, or
 *               det(M) <= 1e-12 (tr(M)/dim)^dim with M = sum dx dx^T).
 *   lambda_out  nullable device out [n_nodes] double: lambda_max of C.
 *   workspace   device, ftle_workspace_bytes(n_nodes) bytes (required).
 * For FP32/FP32C the gradient runs in float; nodes where float loses the result (lambda_max
 * close to 1, two nearly equal top eigenvalues in 3D, an ill-conditioned M) are listed in the
 * workspace and recomputed in FP64 by a second kernel in the same call (or, with
 * ftle_options.defer_fp64, by the ftle_refine that follows). */
int ftle_gradient_eig(const ftle_mesh* mesh, const void* flowmap, int32_t precision, double T,
                      void* ftle_out, double* lambda_out, void* workspace, size_t workspace_bytes,
                      const ftle_options* opt, void* stream);

/* FP32C only (no-op for other precisions): re-advects in float-float arithmetic (~48 bits, on
 * the FP32 pipes) the nodes listed by the last ftle_gradient_eig on this workspace together
 * with their neighbours, writes their flowmap back as (hi, lo) pairs, and recomputes the listed
 * nodes' FTLE in FP64.  For the 2D double gyre and the 3D ABC flow a node's horizon is split into
 * runs integrated side by side and joined through each run's tangent.  Must follow
 * ftle_gradient_eig on the same stream, mesh, flowmap and workspace. */
int ftle_refine(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt,
                int32_t precision, void* flowmap, void* ftle_out, double* lambda_out,
                void* workspace, size_t workspace_bytes, const ftle_options* opt, void* stream);

/* Whole path: ftle_advect, ftle_gradient_eig, then ftle_refine (FP32C).  flowmap is a caller
 * buffer of ftle_flowmap_bytes bytes, left holding the (refined) flowmap. */
int ftle_compute(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt,
                 int32_t precision, void* flowmap, void* ftle_out, double* lambda_out,
                 void* workspace, size_t workspace_bytes, const ftle_options* opt, void* stream);

/* End-to-end from HOST buffers: copies coords (float, or double for FP64), row_ptr and col_idx
 * from host memory into `device_ws`, runs ftle_compute, copies the FTLE field back into
 * ftle_host (float, or double for FP64) and synchronises `stream` before returning.  The
 * copied lists always go through ftle_validate_mesh (on a second stream, while the advection
 * runs): an index out of range returns FTLE_EINVAL before any kernel reads through it.
 * Page-locked host buffers that the device can address (cudaHostAlloc, cudaMallocHost or
 * cudaHostRegister with mapping) are used in place where that saves a copy: for FP32C the
 * advection reads coords_host directly over the host link, and the kernels write the FTLE into
 * ftle_host directly; other buffers (pageable memory) are staged through device_ws by copies.
 * device_ws must hold
 * ftle_host_workspace_bytes(dim, n_nodes, nnz, precision) bytes. */
size_t ftle_host_workspace_bytes(int32_t dim, int64_t n_nodes, int64_t nnz, int32_t precision);
int ftle_compute_host(int32_t dim, int64_t n_nodes, int64_t nnz, const void* coords_host,
                      const int32_t* row_ptr_host, const int32_t* col_idx_host,
                      const ftle_flow* flow, double t0, double T, double dt, int32_t precision,
                      void* ftle_host, void* device_ws, size_t device_ws_bytes,
                      const ftle_options* opt, void* stream);

/* Fixed-width neighbour list from the CSR rows of `mesh` into ell_idx ([width][n_nodes] int32,
 * device, caller-owned), -1 padded.  Reads row_ptr back to the host to check that no row is
 * longer than `width` (FTLE_ERANGE otherwise; nothing launched), then fills ell_idx on `stream`. */
int ftle_ell_from_csr(const ftle_mesh* mesh, int32_t width, int32_t* ell_idx, void* stream);

/* CSR neighbour lists built on the device from element connectivity (NEXT to the paper's host
 * precomputation, Section 2.2, which names accelerating it as future work): nodes a != b are
 * neighbours when some element lists both.  Rows come out sorted, symmetric and without the
 * node itself, as the FTLE kernels expect.
 *   elems      device int32 [n_elem][verts_per_elem] (2 = edges, 3 = triangles, 4 = tetrahedra)
 *   max_row    bound on the raw entries of one node: (verts_per_elem - 1) x the number of elements
 *              touching it (e.g. 3 x 24 for a Kuhn tetrahedral lattice)
 *   row_ptr    device out [n_nodes + 1]; col_idx device out with room for nnz_cap entries
 *   nnz_out    host out: the number of neighbour entries written
 *   workspace  ftle_csr_workspace_bytes(n_nodes, max_row) bytes, 256-byte aligned
 * Synchronous (returns after the lists are complete).  Errors: FTLE_EINVAL when an element names
 * a vertex outside [0, n_nodes) (counted on the device, the element skipped); FTLE_ERANGE when a
 * node exceeds max_row raw entries or nnz exceeds nnz_cap. */
size_t ftle_csr_workspace_bytes(int64_t n_nodes, int32_t max_row);
int ftle_csr_from_elements(int64_t n_nodes, int64_t n_elem, int32_t verts_per_elem, const int32_t* elems,
                           int32_t max_row, int32_t* row_ptr, int32_t* col_idx, int64_t nnz_cap,
                           int64_t* nnz_out, void* workspace, size_t workspace_bytes, void* stream);

/* Validation of a mesh's neighbour lists, the contract of the paper's host-side neighbour
 * precomputation (Section 2.2): the FTLE core gathers coordinates and flowmaps through these
 * indices, so every one must name a node.  One pass on the device reads row_ptr, col_idx and
 * (when set) ell_idx and checks, without dereferencing any value it reads:
 *   row_ptr[0] = 0, row_ptr non-decreasing, row_ptr[n_nodes] = nnz;
 *   0 <= col_idx[e] < n_nodes for every e < nnz;
 *   -1 <= ell_idx[t] < n_nodes for every t < ell_width * n_nodes.
 *   report     nullable HOST out: how many entries of each array are bad and the position of the
 *              first (-1 when none).
 *   workspace  device, >= 256 bytes, 256-byte aligned; bytes 128..175 are overwritten (the start
 *              of a ftle_workspace_bytes workspace serves, its counters stay as they were).
 * Synchronous: waits for `stream`.  Returns FTLE_EINVAL (message naming the first bad entry)
 * when any check fails, FTLE_OK otherwise.  The other entry points check sizes and pointers on
 * the host but trust the index values; they run this pass themselves when
 * ftle_options.validate_mesh = 1 (ftle_compute_host always does). */
typedef struct ftle_mesh_report {
  int64_t bad_row_ptr;    /* rows i with row_ptr[i+1] < row_ptr[i], row_ptr[0] != 0 (row 0) or
                             row_ptr[n_nodes] != nnz (row n_nodes - 1) */
  int64_t bad_col_idx;    /* col_idx entries outside [0, n_nodes) */
  int64_t bad_ell_idx;    /* ell_idx entries outside [-1, n_nodes) */
  int64_t first_bad_row;  /* lowest such row, -1 if none */
  int64_t first_bad_col;  /* lowest such col_idx position, -1 if none */
  int64_t first_bad_ell;  /* lowest such ell_idx position (s * n_nodes + i), -1 if none */
} ftle_mesh_report;
int ftle_validate_mesh(const ftle_mesh* mesh, ftle_mesh_report* report, void* workspace,
                       size_t workspace_bytes, void* stream);

/* Synchronous read of the counters at the start of `workspace` (waits for `stream`). */
int ftle_read_counters(const void* workspace, ftle_counters* out, void* stream);

/* FTLE core with no device allocation anywhere, for callers that may not allocate.  The paper
 * has no counterpart; this is a service of the library.  Some callers cannot hand the library a
 * workspace: a plugin whose host application owns every device allocation, a component that runs
 * under a fixed device-memory budget fixed at start-up, or a latency-critical loop that must not
 * call cudaMalloc / cudaFree (cudaFree can synchronise the whole device).  This entry point does
 * the work of ftle_gradient_eig with its scratch (the counters and the list of nodes that take
 * the FP64 path) in a file-scope device array of the library instead of a caller workspace.
 *   - Limit: n_nodes <= FTLE_NOALLOC_MAX_NODES; larger meshes return FTLE_ERANGE, nothing launched.
 *   - Memory: the array (FTLE_NOALLOC_MAX_NODES * 4 + 256 bytes, about 4 MiB) is part of the
 *     library's device image, so every GPU that loads libftle.so holds it until the process exits.
 *   - Set-up: a call outside stream capture looks up the array's device address
 *     (cudaGetSymbolAddress) with the calling device current; a call on a capturing stream reuses
 *     the address from the last call on that device outside capture.  So make the first call on
 *     each device before any stream capture begins there (a first call inside a capture returns
 *     FTLE_EINVAL), and after a cudaDeviceReset make one call outside capture before capturing
 *     again.
 *   - Sharing: all calls share the one array, and each call clears the counters it needs at its
 *     start (the array keeps the last call's contents otherwise).  Two calls whose work overlaps
 *     on the GPU (for example on two streams) race on the array and corrupt each other's FP64
 *     node list; serialise them.
 *   - Arguments, outputs and errors otherwise as ftle_gradient_eig (flowmap, ftle_out and
 *     lambda_out are caller device buffers; no counters are returned), except that the FP64 pass
 *     of the flagged nodes always runs inside this call: ftle_options.defer_fp64 = 1 returns
 *     FTLE_EINVAL, and no ftle_refine can follow this call (its flag list lives in the array,
 *     not in a workspace an ftle_refine could be given). */
#define FTLE_NOALLOC_MAX_NODES 1048576
int ftle_gradient_eig_noalloc(const ftle_mesh* mesh, const void* flowmap, int32_t precision, double T,
                              void* ftle_out, double* lambda_out, const ftle_options* opt,
                              void* stream);

/* ---------------------------------------------------------------------------------- batched */

/* Many independent problems of uneven size and horizon in one launch sequence: one persistent
 * advection kernel and one persistent gradient kernel walk a shared queue of (instance, tile)
 * items ordered longest-first (LPT), followed by the FP64 fix-up of flagged nodes.  All
 * instances share dt and precision (FP32 or FP32C); per-instance t0 = 0.
 *   meshes, flows, T  HOST arrays [n_inst] (mesh pointers inside are device pointers).
 *   ftle_out          HOST array [n_inst] of device float pointers [meshes[i].n_nodes].
 *   workspace         device, ftle_batch_workspace_bytes(...) bytes, 256-byte aligned. */
size_t ftle_batch_workspace_bytes(int32_t n_inst, const ftle_mesh* meshes, int32_t precision);
int ftle_batch(int32_t n_inst, const ftle_mesh* meshes, const ftle_flow* flows, const double* T,
               double dt, int32_t precision, void* const* ftle_out, void* workspace,
               size_t workspace_bytes, const ftle_options* opt, void* stream);

/* A batch captured once into a CUDA graph and replayed: create builds the queue, uploads it
 * into the workspace and captures the kernels; launch replays the graph on `stream`; destroy
 * frees the graph.  The buffers named at create time must stay valid while the plan lives. */
typedef struct ftle_batch_plan ftle_batch_plan;
int ftle_batch_plan_create(int32_t n_inst, const ftle_mesh* meshes, const ftle_flow* flows,
                           const double* T, double dt, int32_t precision, void* const* ftle_out,
                           void* workspace, size_t workspace_bytes, const ftle_options* opt,
                           void* stream, ftle_batch_plan** plan);
int ftle_batch_plan_launch(ftle_batch_plan* plan, void* stream);
int ftle_batch_plan_destroy(ftle_batch_plan* plan);

/* ----------------------------------------------------------------------------- differentiation */

/* Reverse-mode derivative of L = sum_i dL_dftle[i] FTLE_i with respect to the double-gyre
 * parameters (A, eps, omega), 2D, FP32/FP32C forward.  Steps: the adjoint of the FTLE map gives
 * dL/dphi at every node (a gather over the symmetric adjacency; the CSR lists must be
 * symmetric), then the discrete adjoint of the RK4 steps runs backward segment by segment,
 * recomputing each segment's states from the checkpoints written by ftle_advect, and the
 * per-step parameter terms are summed in FP64 in a fixed order (deterministic).
 *   flowmap, checkpoints  as written by ftle_advect with the same arguments and ckpt_every.
 *   dL_dftle              device float [n_nodes].
 *   dL_dparams            device double [3] out.
 *   workspace             ftle_backward_workspace_bytes(n_nodes, dim) bytes. */
size_t ftle_backward_workspace_bytes(int64_t n_nodes, int32_t dim);
int ftle_backward(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt,
                  int32_t precision, const void* flowmap, const void* checkpoints,
                  int32_t ckpt_every, const float* dL_dftle, double* dL_dparams, void* workspace,
                  size_t workspace_bytes, const ftle_options* opt, void* stream);

/* ---------------------------------------------------------------------------------- misc */

const char* ftle_status_string(int status);
const char* ftle_last_error(void); /* message of the calling thread's last failing call */
int ftle_version(void);            /* FTLE_API_VERSION */

#ifdef __cplusplus
}
#endif

#endif /* FTLE_H */
