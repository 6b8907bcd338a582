// Internal data structures of the fsim library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/fsim.h"

namespace fsim {

// ---------------------------------------------------------------------------
// Host-side precomputation results (prefactor.cpp)
// ---------------------------------------------------------------------------
struct Supernode {
  int c0 = 0, ns = 0;           // first solver position and number of columns
  int nr1 = 0;                  // off-diagonal rows inside x1
  int nr = 0;                   // all off-diagonal rows kept (x1 rows, then x2 rows)
  int64_t rows_off = 0;         // offset of its nr1 row positions in rows[]
  int64_t z_off = 0;            // offset of its Z block ((ns+nr) x ns, col-major)
  int level = 0;                // 0 = leaf; parents have larger levels
};

struct HostFactor {
  int n_free = 0, n1 = 0, n2 = 0;
  std::vector<int> perm;        // solver position -> mesh vertex (x1 then x2)
  std::vector<int> pos;         // mesh vertex -> solver position or -1 (pinned)
  std::vector<Supernode> sn;    // post-ordered supernodes of L11
  std::vector<int> rows;        // off-diagonal row positions (x1 and x2) per supernode
  std::vector<double> Z;        // per supernode [L_JJ^-1 ; L_RJ L_JJ^-1]
  std::vector<int> level_ptr;   // supernodes grouped by level (CSR)
  std::vector<int> level_sn;
  int n_levels = 0;
  // couplings (solver positions): K12 rows x1 -> cols x2 (col index - n1),
  // K21 rows x2 -> cols x1
  std::vector<int> k12_ptr, k12_col; std::vector<double> k12_val;
  std::vector<int> k21_ptr, k21_col; std::vector<double> k21_val;
  // full free-DOF K (solver positions) for residual checks / refinement
  std::vector<int> k_ptr, k_col; std::vector<double> k_val;
  std::vector<double> sigma_inv;  // n2 x n2 dense, row-major (symmetric)
  std::vector<double> sigma;      // n2 x n2 Sigma, row-major (symmetric)
  double kappa_auto = 0.0;        // mean diag(H) over free DOFs
  int64_t factor_nnz = 0;
};

// Per-tet rest data computed on the host (w and Dm^-1).
void tet_rest_data(const double* rest, const int32_t* tets, int64_t T, double weight_scale,
                   std::vector<double>& dminv /*9T SoA*/, std::vector<double>& w);

// Build K, the ordering, the factor of K11 and Sigma^-1.  Returns an fsim status.
int build_factor(int64_t n, const double* rest, const int32_t* tets, int64_t T,
                 const std::vector<double>& dminv, const std::vector<double>& w,
                 const uint8_t* pinned, const std::vector<uint8_t>& x2mask,
                 HostFactor& f);

}  // namespace fsim
