// Gaussian-well potential on the helical grid, summed over the images of the symmetry group
// (arXiv 2210.12252, eqs. symm_opera and sim_atoms; V obeys eq. Potential_Symmetry by
// construction):
//
//   V(x) = sum_a sum_{zeta, mu} -Z_a exp(-|x - Upsilon_{zeta,mu} x_a|^2 / (2 sigma_a^2)),
//   Upsilon_{zeta,mu}: rotation by 2 pi zeta alpha + 2 pi mu / Ncyc about e_Z, then zeta tau e_Z,
//
// keeping the images with |z - z_image| <= 10 sigma.  Grid points map to cylindrical
// coordinates by inverting eq. coordinates_conversion (z = tau theta1,
// vartheta = 2 pi (theta2 + alpha theta1)).  Output in eq. wavefun_storage_real order.
//
// This is the once-per-potential setup step; it runs in FP64 on the host's cores (std::thread
// over theta1 planes): on this GPU FP64 exponentials are slower than on the host.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "hw_internal.h"

namespace hw {

void build_gaussian_potential(const HostBasis& hb, int n_atoms, const double* atoms,
                              std::vector<double>& V) {
  const auto& p = hb.prm;
  const int n1 = p.Nth1, n2 = p.Nth2, nr = p.Nr;
  V.assign((size_t)n1 * n2 * nr, 0.0);
  const double pi = 3.14159265358979323846;
  auto work = [&](int i0, int i1) {
    for (int i = i0; i < i1; ++i) {
      const double th1 = double(i) / n1;
      const double z = p.tau * th1;
      for (int a = 0; a < n_atoms; ++a) {
        const double ra = atoms[5 * a], tha = atoms[5 * a + 1], za = atoms[5 * a + 2];
        const double Z = atoms[5 * a + 3], sig = atoms[5 * a + 4];
        const double cut = 10.0 * sig, inv2s2 = 1.0 / (2.0 * sig * sig);
        const int zlo = (int)std::floor((z - cut - za) / p.tau);
        const int zhi = (int)std::ceil((z + cut - za) / p.tau);
        for (int zeta = zlo; zeta <= zhi; ++zeta) {
          const double dz = z - (za + zeta * p.tau);
          if (std::fabs(dz) > cut) continue;
          for (int mu = 0; mu < p.ncyc; ++mu) {
            const double ang = tha + 2.0 * pi * zeta * p.alpha + 2.0 * pi * mu / p.ncyc;
            for (int j = 0; j < n2; ++j) {
              const double vth = 2.0 * pi * (double(j) / (p.ncyc * n2) + p.alpha * th1);
              const double cs = std::cos(vth - ang);
              double* out = &V[((size_t)i * n2 + j) * nr];
              for (int q = 0; q < nr; ++q) {
                const double r = hb.r[q];
                const double d2 = r * r + ra * ra - 2.0 * r * ra * cs + dz * dz;
                out[q] += -Z * std::exp(-d2 * inv2s2);
              }
            }
          }
        }
      }
    }
  };
  unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  nt = std::min<unsigned>(nt, (unsigned)n1);
  std::vector<std::thread> th;
  const int per = (n1 + (int)nt - 1) / (int)nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int i0 = (int)t * per, i1 = std::min(n1, i0 + per);
    if (i0 < i1) th.emplace_back(work, i0, i1);
  }
  for (auto& t : th) t.join();
}

}  // namespace hw
