// Internal declarations shared by the host runtime and the CUDA kernels of
// the spaND library.  Nothing here crosses the C ABI.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace spand {

// Symbolic structure of one elimination step (all indices into the step's
// cluster list).
struct StepStruct {
  int n = 0;
  std::vector<int32_t> keys;                 // 3 n: S, L, R heap labels
  std::vector<int32_t> child_ptr, child_idx; // into the previous step's list
  std::vector<int32_t> elim;                 // 1 = eliminated at this step
  std::vector<int32_t> colour;               // -1 for eliminated clusters
  std::vector<int32_t> adj_ptr, adj_idx;     // cluster graph before the step
  std::vector<int32_t> adjf_ptr, adjf_idx;   // remaining clusters after fill
  int ncolours() const {
    int c = 0;
    for (int32_t v : colour) c = v + 1 > c ? v + 1 : c;
    return c;
  }
};

struct Tree {
  int64_t n = 0;
  int L = 0;
  std::vector<int32_t> perm;         // perm[i] = vertex at position i
  std::vector<int32_t> cluster_ptr;  // n_clusters + 1
  std::vector<int32_t> keys;         // 3 per cluster
  std::vector<StepStruct> steps;     // L steps
};

int analyze_tree(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* coords,
                 int dim, int L, Tree& T, std::string& err);
int validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colind, std::string& err);

}  // namespace spand
