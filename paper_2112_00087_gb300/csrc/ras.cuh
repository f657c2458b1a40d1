// Restricted additive Schwarz preconditioner (internal interface).
#pragma once

#include "common.cuh"

namespace helm {

struct RasPrecond;

// Interface (Robin) coefficients of the subdomain matrices: lo on the low faces of each extended
// box (planes i0, j0, l0), hi on its high faces; per_h: each face's coefficient divided by the
// lattice spacing normal to it. Zero for plain RAS.
struct RasRobin {
  cd lo = cd(0.0, 0.0), hi = cd(0.0, 0.0);
  bool per_h = false;
};

// Partition the lattice into parts[0] x parts[1] x parts[2] owned blocks (node (i,j,l) belongs
// to block (floor(i P_x / (nx+1)), ...)), extend each by `overlap` lattice layers, extract the
// subdomain matrices A_s = R_s A R_s^T from the CSR matrix, add the Robin terms of `robin` (face
// mass of the extended box's faces inside the lattice, Dirichlet nodes excluded; optimized
// Schwarz interface terms) when they are non-zero, and factor them (banded LDL^T, complex
// symmetric, no pivoting) on stream s. Synchronises s.
helm_status ras_create(const helm_ctx* ctx, const int32_t* rowptr, const int32_t* col, const cd* val,
                       const int32_t parts[3], int overlap, const RasRobin& robin, RasPrecond** out,
                       cudaStream_t s);
// out = sum_s Rt_s^T A_s^-1 R_s in (ordered on stream s, capturable). The kernel returns at
// once when *skip_a or *skip_b (device flags, may be null) is non-zero.
helm_status ras_apply(RasPrecond* P, const cd* in, cd* out, const int* skip_a, const int* skip_b,
                      cudaStream_t s);
// HELM_PIVOT if a factorisation met a pivot below 1e-12 max|diag| (synchronises).
helm_status ras_status(RasPrecond* P);
void ras_destroy(RasPrecond* P);

}  // namespace helm
