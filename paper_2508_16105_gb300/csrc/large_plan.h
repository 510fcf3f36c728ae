// Gather plan of the CTA-per-cell kernel (large mechanisms).
//
// Built on the host from the packed mechanism image, uploaded once behind it.
// Every quantity the block accumulates over reactions is listed per output, in
// ascending reaction order, so each output is one thread's fixed-order sum:
//   omega_k     = sum_{e in spr[k]} nu_e q_{r_e}                 (also d omega_k / dT)
//   D[k][j]     = A_k + sum_{q in ent(k,j)} coef_q RS[r_q][slot_q]
//   A_k         = sum_{e in row[k]} nu_e allc_{r_e}              (third-body / falloff [M] term, all j)
// where RS[r] holds the reaction's per-side derivatives (slots 0-2 forward, 3-5
// reverse), d q / d[M] (slot 6), q (slot 7) and d q / dT (slot 8).
//
// The plan also carries a compact per-reaction table as structure of arrays
// (ln A, b, E/R, sum of net coefficients; one int4 of packed integers), which the
// kernel stages in shared memory so that consecutive threads read consecutive
// reactions.  Packed integers:
//   x: type (bits 0-1) | reversible (bit 2) | nf (bits 3-4) | nb (bits 5-6) |
//      forward orders (2 bits each from bit 8) | reverse orders (2 bits each from bit 14)
//   y: forward species (10 bits each), z: reverse species (10 bits each), w: spare
#pragma once
#include <stdint.h>

namespace rde {

struct PlanHeader {
  int32_t K, R, n_spr, n_ent, n_con, n_row, bytes, pad;
  // byte offsets of the arrays from the start of the plan (each 16-byte aligned)
  int32_t o_spr_ptr, o_spr_r, o_spr_nu, o_ent_index, o_ent_ptr, o_con_r, o_con_slot, o_con_coef, o_row_ptr, o_row_r,
      o_row_nu, o_rx;
  // o_rx: the reaction table, one contiguous block of rx_bytes:
  //   lnA[R], b[R], EaR[R], dnu[R] (doubles, R rounded up to an even count), meta[R] (int4)
  int32_t rx_bytes, rx_stride, pad2[2];
};
static_assert(sizeof(PlanHeader) % 16 == 0, "plan header alignment");

struct PlanView {
  const int32_t* spr_ptr;   // K + 1
  const int32_t* spr_r;     // n_spr
  const double* spr_nu;     // n_spr
  const int32_t* ent_index; // K * K: entry id of (k, j) or -1
  const int32_t* ent_ptr;   // n_ent + 1
  const int32_t* con_r;     // n_con
  const int32_t* con_slot;  // n_con
  const double* con_coef;   // n_con
  const int32_t* row_ptr;   // K + 1
  const int32_t* row_r;     // n_row
  const double* row_nu;     // n_row
};

// Doubles per array of the reaction table (R rounded up so the int4 block stays 16-byte aligned).
#if defined(__CUDACC__)
__host__ __device__ __forceinline__
#else
inline
#endif
int plan_rx_stride(int R) { return (R + 1) & ~1; }

#if defined(__CUDACC__)
__host__ __device__ __forceinline__
#else
inline
#endif
int plan_rx_bytes(int R) { return 4 * 8 * plan_rx_stride(R) + 16 * R; }

#if defined(__CUDACC__)
__host__ __device__ __forceinline__
#else
inline
#endif
PlanView plan_view(const unsigned char* plan) {
  const PlanHeader* h = reinterpret_cast<const PlanHeader*>(plan);
  PlanView v;
  v.spr_ptr = reinterpret_cast<const int32_t*>(plan + h->o_spr_ptr);
  v.spr_r = reinterpret_cast<const int32_t*>(plan + h->o_spr_r);
  v.spr_nu = reinterpret_cast<const double*>(plan + h->o_spr_nu);
  v.ent_index = reinterpret_cast<const int32_t*>(plan + h->o_ent_index);
  v.ent_ptr = reinterpret_cast<const int32_t*>(plan + h->o_ent_ptr);
  v.con_r = reinterpret_cast<const int32_t*>(plan + h->o_con_r);
  v.con_slot = reinterpret_cast<const int32_t*>(plan + h->o_con_slot);
  v.con_coef = reinterpret_cast<const double*>(plan + h->o_con_coef);
  v.row_ptr = reinterpret_cast<const int32_t*>(plan + h->o_row_ptr);
  v.row_r = reinterpret_cast<const int32_t*>(plan + h->o_row_r);
  v.row_nu = reinterpret_cast<const double*>(plan + h->o_row_nu);
  return v;
}

}  // namespace rde
