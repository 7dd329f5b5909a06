// specialize.h -- mechanism-specialised integration kernels, compiled at run time.
//
// The integration kernels (integrate.cuh) take the mechanism's sizes (species, reactions, nonzeros, program
// steps) and the cell layout's offsets from by-value views.  For one mechanism these are constants: the
// run-time compiler (NVRTC) builds the one-warp-per-cell kernels again with views whose sizes and offsets
// are compile-time constants, so that loop trip counts and shared-memory addresses fold into the code.
// The data members stay those of MechView / CellLayout, so the host passes the same objects.
#pragma once
#include <string>

#include "../../include/chem.h"
#include "compile.h"

namespace chemgb {

struct SpecKernels {
  void* library[2] = {nullptr, nullptr};   // cudaLibrary_t of the plain and the persistent kernel
  const void* plain = nullptr;             // cudaKernel_t, usable wherever a kernel's host handle is
  const void* persistent = nullptr;
  double compile_s = 0.0;                  // wall time of the compilation (0 when both came from the cache)
  bool from_cache = false;
};

// Source of the specialised instantiation for mechanism hm with cell layout L (lane group: one warp).
std::string specialized_source(const HostMech& hm, const CellLayout& L);

// Compile (or take from the on-disk cache) both kernels and, when load is set, load them into the current
// device's context (load false: only fill the cache; no CUDA call).  CHEM_EUNSUPPORTED when the run-time
// compiler cannot be loaded; CHEM_ECUDA when compiling or loading fails (err holds the compiler's log).
chem_status compile_specialized(const HostMech& hm, const CellLayout& L, bool load, SpecKernels& out,
                                std::string& err);

void release_specialized(SpecKernels& k);

}  // namespace chemgb
