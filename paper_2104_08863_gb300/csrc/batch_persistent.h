// Device-side records of the persistent batched launch (batch_persistent.cu) and its host hooks.
#pragma once

#include "internal.h"

namespace pp {

enum BatchPass : int { BP_XF = 0, BP_ZF = 1, BP_TRI = 2, BP_LOW = 3, BP_ZI = 4, BP_XI = 5, BP_N = 6 };

// One instance of the batch, as the persistent kernel reads it.
struct BatchInst {
  Geometry g;
  DevTables dt;            // table pointers into the instance's workspace
  cplx<float>* spec;       // the instance's spectral buffer
  const float* rhs;        // caller's right-hand side and result (set per pointer set)
  float* out;
  double* low_piv;         // FP64 scratch of the low modes: pivots [row][system]
  cplx<double>* low_y;     //   and forward values [row][system]
  int parts, low;          // PDD blocks per system, low-mode half-width
  int xsel, zsel, msel;    // selectors of the specialised tile functions
  int zcols;               // z-transform tiles per y-plane
  int ntiles[BP_N];        // tiles of each pass
};

// Tiles tile .. tile + count - 1 of one pass of one instance.
struct BatchItem {
  int inst, pass, tile, count;
};

// Control block, cleared before every launch.
struct BatchCtl {
  unsigned ticket;
  unsigned abort;
  unsigned done[1];        // [instance][pass] counters (allocated for the whole batch)
};

int batch_persistent_smem();
bool batch_persistent_ok(const poisson_plan_s* c, int& xsel, int& zsel, int& msel);
void batch_tiles(const poisson_plan_s* c, int zcols, int ntiles[BP_N]);
int batch_group(const poisson_plan_s* c, int pass, int zcols);
int batch_zcols(const poisson_plan_s* c);
cudaError_t launch_batch_persistent(const BatchInst* inst, const BatchItem* items, int nitems, BatchCtl* ctl,
                                    size_t ctl_bytes, int* status, int selftest, cudaStream_t st);

}  // namespace pp
