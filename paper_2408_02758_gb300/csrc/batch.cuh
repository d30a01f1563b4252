// Batched execution: many independent FTLE problems (uneven meshes and horizons) walked by
// persistent kernels through a queue of (instance, node range) items.
#pragma once

#include "advect.cuh"
#include "gradient.cuh"

namespace ftle {

struct BatchInst {
  AdvArgs adv;   // advection arguments of this instance (coords, flowmap, step, parameters)
  GradArgs grad; // gradient arguments (CSR, flowmap, FTLE output, 1/(2|T|), batch counters)
  int64_t off;   // first index of this instance in the batch-wide node numbering (mark bitmap)
};

struct BatchItem {
  int32_t inst, lo, hi, pad;  // nodes [lo, hi) of instance inst
};

// Batch-wide counters: ftle_counters at offset 0 of the workspace, whose reserved words hold the
// two queue heads.
struct BatchQueues {
  unsigned int* adv_next;
  unsigned int* grad_next;
};

int launch_batch_advect(int kind, int dim, int prec, const BatchInst* insts, const BatchItem* items,
                        int n_items, unsigned int* next, int grid, int block, size_t smem, cudaStream_t s);
int launch_batch_grad(int dim, int phi_layout, const BatchInst* insts, const BatchItem* items, int n_items,
                      unsigned int* next, ftle_counters* hdr, int2* flags, int grid, int block, cudaStream_t s);
int launch_batch_grad_f64(int dim, int phi_layout, const BatchInst* insts, const int2* pairs,
                          const unsigned long long* count, int grid, int block, cudaStream_t s);
int launch_batch_mark(const BatchInst* insts, const int2* flags, const unsigned long long* n_flags, int2* marks,
                      unsigned long long* n_marks, uint32_t* bitmap, int grid, int block, cudaStream_t s);
// Run-parallel batched re-advection of compensated 2D double-gyre instances (every instance's
// flowmap carries its run-boundary states).
int launch_batch_refine_runs_dg(const BatchInst* insts, const int2* pairs, const unsigned long long* count, int grid,
                                cudaStream_t s);
int launch_batch_advect_ds(int kind, int dim, const BatchInst* insts, const int2* pairs,
                           const unsigned long long* count, int grid, int block, cudaStream_t s);

}  // namespace ftle
