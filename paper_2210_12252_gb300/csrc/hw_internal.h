// Internal definitions shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/helicwave.h"

namespace hw {

// ------------------------------------------------------------------ host-side basis data
struct HostBasis {
  hw_basis_params prm{};
  int M = 0, N = 0, K = 0;
  std::vector<double> r, wr;                 // [Nr] radial nodes / weights (int f r dr)
  std::vector<std::vector<double>> zeros;    // zeros[|n|][k]: b_k^{|n| Ncyc}
  std::vector<double> xi;                    // [(N+1)][Nr][K]: xi_{n,k}(r_p), n >= 0
  std::vector<double> qtab;                  // [(N+1)][K][K]: <F_{m,n,k'}, F_{m,n,k} / r^2>
  std::vector<double> xid;                   // [(N+1)][Nr][K]: d xi_{n,k} / dr at r_p
  // k-points
  int nk = 0;
  std::vector<double> eta, nu, ecut;
  std::vector<int64_t> L;                    // [nk] kept modes
  // angular pairs kept at any k-point, grouped by |n| (table index), then n, then m
  int nA = 0;
  std::vector<int> pair_m, pair_n;           // [nA]
  std::vector<int> group_start;              // [N+2]: pairs of |n| = g are [gs[g], gs[g+1])
  std::vector<int> mrow_m;                   // active m values (ascending)
  std::vector<int> pair_mrow;                // [nA] index into mrow_m
  std::vector<int> slot_pair;                // [nmr][Nth2]: the pair at (m row, n mod Nth2), or -1
  // per k-point / per pair: compact offset and kept radial count
  std::vector<int> off;                      // [nk][nA]
  std::vector<int> Ka;                       // [nk][nA]
  std::vector<std::vector<double>> ke;       // [nk][L]: shifted kinetic energy, compact order
  std::vector<std::vector<int32_t>> mnk;     // [nk][3L]
};

// Build everything above.  Returns an empty string on success, else the error message.
std::string build_host_basis(const hw_basis_params& p, int nk, const double* eta,
                             const double* nu, const double* ecut_per_k, HostBasis& hb);

// FFT plan for one length (radices 4, 3, 2 in stage order).
struct FftPlan {
  int n = 0;
  int nst = 0;
  int rad[16] = {0};
};
bool make_fft_plan(int n, FftPlan& plan);

}  // namespace hw

namespace hw {
// Gaussian-well potential (host, FP64) in eq. wavefun_storage_real order; atoms [n][5] =
// (r, vartheta, z, Z, sigma).
void build_gaussian_potential(const HostBasis& hb, int n_atoms, const double* atoms,
                              std::vector<double>& V);
}  // namespace hw
