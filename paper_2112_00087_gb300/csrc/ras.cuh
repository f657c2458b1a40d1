// Restricted additive Schwarz preconditioner (internal interface).
#pragma once

#include "common.cuh"

namespace helm {

struct RasPrecond;

// Partition the lattice into parts[0] x parts[1] x parts[2] owned blocks (node (i,j,l) belongs
// to block (floor(i P_x / (nx+1)), ...)), extend each by `overlap` lattice layers, extract the
// subdomain matrices A_s = R_s A R_s^T from the CSR matrix, add robin * (face mass of the
// extended box's faces inside the lattice, Dirichlet nodes excluded) when robin != 0 (optimized
// Schwarz interface term), and factor them (banded LDL^T, complex symmetric, no pivoting) on
// stream s. Synchronises s.
helm_status ras_create(const helm_ctx* ctx, const int32_t* rowptr, const int32_t* col, const cd* val,
                       const int32_t parts[3], int overlap, cd robin, RasPrecond** out, cudaStream_t s);
// out = sum_s Rt_s^T A_s^-1 R_s in (ordered on stream s, capturable). The kernel returns at
// once when *skip_a or *skip_b (device flags, may be null) is non-zero.
helm_status ras_apply(RasPrecond* P, const cd* in, cd* out, const int* skip_a, const int* skip_b,
                      cudaStream_t s);
// HELM_PIVOT if a factorisation met a pivot below 1e-12 max|diag| (synchronises).
helm_status ras_status(RasPrecond* P);
void ras_destroy(RasPrecond* P);

}  // namespace helm
