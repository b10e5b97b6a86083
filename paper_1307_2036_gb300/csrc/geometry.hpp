// Host-side construction of the grid hierarchy: per-level column metrics and
// connectivity, and the per-problem radial vectors.  FP64 throughout; the
// device keeps FP64 and FP32 copies.
#pragma once

#include <cstdint>
#include <vector>

namespace ells {

struct HostLevel {
    int n = 0;                  // cells per panel side
    int64_t ncol = 0;           // P * n * n
    std::vector<double> area;   // [ncol] cell area (unit sphere, or flat box)
    std::vector<double> trans;  // [ncol*4] face length / centre distance, faces -i,+i,-j,+j
    std::vector<int32_t> nbr;   // [ncol*4] neighbouring column across each face
    std::vector<int32_t> pst;   // [ncol*4] prolongation stencil from the next coarser
                                //          level: parent, x-neighbour, y-neighbour,
                                //          diagonal (-1 where three cells meet)
};

struct HostHierarchy {
    int kind = 0, P = 1, mapping = 0;
    double side = 0.0;
    std::vector<HostLevel> levels;  // 0 = finest
};

// Build all levels: halve n while n is even and n/2 >= coarsest_min, at most
// max_levels levels (<= 0: no cap).
HostHierarchy build_hierarchy(int kind, int n, int mapping, double side, int coarsest_min,
                              int max_levels);

// Radial vectors of the shell r_0 < ... < r_nz:
//   V[k] = int_{r_k}^{r_{k+1}} r^2 dr                      (k < nz)
//   G[k] = r_k^2 / (rho_k - rho_{k-1}), rho_k cell centres  (0 < k < nz), G[0] = G[nz] = 0
void radial_vectors(const double *r, int nz, std::vector<double> &V, std::vector<double> &G);

}  // namespace ells
