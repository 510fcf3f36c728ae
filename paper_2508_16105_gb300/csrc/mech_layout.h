// Packed mechanism tables shared by the host packer and the device kernels.
//
// A loaded mechanism becomes one contiguous, 16-byte aligned byte image:
//   [MechHeader][SpecPacked x K][RxnPacked x R][EffEntry x n_eff]
//   [exp table: 1024 doubles][log table: 128 (invc, logc) pairs]
// The kernels copy the image into shared memory once per CTA; every lane of
// a warp then reads the same reaction record at the same time (a broadcast).
//
// Units: SI (mol, m^3, s, K, kg).  Pre-factors are stored as ln A with A
// converted from mol-cm-s by 1e-6 per reaction order above one; activation
// energies as E/R_u in K.
#pragma once
#if !defined(__CUDACC_RTC__)  /* run-time compilation: types from the preamble */
#include <stdint.h>
#endif

namespace rde {

constexpr double kRuHost = 8.31446261815324;  // J/(mol K)
constexpr int kMaxSide = 3;        // distinct species on one side of a reaction
constexpr int kMaxPart = 6;        // distinct species with non-zero net stoichiometry
constexpr int kMaxOrder = 3;       // stoichiometric coefficient of one species on one side

enum RxnType : int32_t { RX_ELEM = 0, RX_THREEBODY = 1, RX_LINDEMANN = 2, RX_TROE = 3 };

struct MechHeader {
  int32_t K, R, n_eff, n_threebody;
  int32_t n_falloff, bytes, tab_offset, pad1;
};

// NASA-7 coefficients re-expressed per temperature range r (0: T < Tmid, 1: T >= Tmid)
//   Cp/R  = cp[r][0] + T (cp[1] + T (cp[2] + T (cp[3] + T cp[4])))
//   H/RT  = h[r][0] + T (h[1] + T (h[2] + T (h[3] + T h[4]))) + h[5] / T
//   G/RT  = H/RT - S/R = g[r][0] + g[r][1] ln T + T (g[2] + T (g[3] + T (g[4] + T g[5]))) + g[6] / T
//   dCp/R/dT = dcp[r][0] + T (dcp[1] + T (dcp[2] + T dcp[3]))
struct SpecPacked {
  double W, Winv, Tmid, pad;
  double cp[2][5];
  double h[2][6];
  double g[2][7];
  double dcp[2][4];
};

struct RxnPacked {
  double lnA, b, EaR;          // k (k_inf for falloff) = exp(lnA + b ln T - EaR / T)
  double lnA0, b0, EaR0;       // k_0 (falloff only)
  double troe_a, troe_invT3, troe_invT1, troe_T2;  // T2 used only if has_T2
  double dnu;                  // sum of net stoichiometric coefficients
  double pnu[kMaxPart];        // net coefficient of each participant
  double fod[kMaxSide], bod[kMaxSide];  // reactant / product orders as doubles
  int32_t type, rev, nf, nb, np, eff_begin, eff_end, has_T2;
  int32_t fi[kMaxSide], fo[kMaxSide];   // reactant species and orders
  int32_t bi[kMaxSide], bo[kMaxSide];   // product species and orders
  int32_t pi[kMaxPart];                 // participants (net coefficient != 0)
};

// third-body efficiency that differs from 1: [M] = sum_k c_k + sum_e (alpha_e - 1) c_{k_e}
struct EffEntry {
  double alpha_minus_1;
  int32_t k, pad;
};

static_assert(sizeof(MechHeader) % 16 == 0, "header alignment");
static_assert(sizeof(SpecPacked) % 16 == 0, "species alignment");
static_assert(sizeof(RxnPacked) % 16 == 0, "reaction alignment");
static_assert(sizeof(EffEntry) % 16 == 0, "efficiency alignment");

struct MechView {
  const MechHeader* hdr;
  const SpecPacked* sp;
  const RxnPacked* rx;
  const EffEntry* eff;
  const double* exptab;   // 2^(j/1024), j < 1024
  const double* logtab;   // (invc_j, logc_j), j < 128
};

#if defined(__CUDACC__)
#define RDE_HD __host__ __device__ __forceinline__
#else
#define RDE_HD inline
#endif

RDE_HD MechView mech_view(const void* image) {
  const char* p = static_cast<const char*>(image);
  MechView v;
  v.hdr = reinterpret_cast<const MechHeader*>(p);
  v.sp = reinterpret_cast<const SpecPacked*>(p + sizeof(MechHeader));
  v.rx = reinterpret_cast<const RxnPacked*>(p + sizeof(MechHeader) + sizeof(SpecPacked) * v.hdr->K);
  v.eff = reinterpret_cast<const EffEntry*>(p + sizeof(MechHeader) + sizeof(SpecPacked) * v.hdr->K +
                                            sizeof(RxnPacked) * v.hdr->R);
  v.exptab = reinterpret_cast<const double*>(p + v.hdr->tab_offset);
  v.logtab = v.exptab + 1024;
  return v;
}

}  // namespace rde
