#pragma once

#include <functional>

namespace gbd {
// f(0..n-1) on the engine's persistent host worker pool (engine.cpp)
void host_parallel_for(int n, const std::function<void(int)>& f);
// Symmetric eigendecomposition of an n x n row-major matrix: eigenvalues
// ascending in w, eigenvector j in column j of Z (row-major n x n).
// Returns 0, or -1 if the QL iteration does not converge.
int sym_eig(int n, const double* A, double* w, double* Z);
// M (m x c, m <= c) = Lo * Q with orthonormal rows written back into M.
int row_orthonormalize(int m, int c, double* M, double* Lo);
}  // namespace gbd
