// Small dense eigenproblems of the restarted Arnoldi eigensolver (host code):
// the m x m projected matrix (m <= 512) in complex Schur form A = Z T Z^H,
// reordered so that the wanted eigenvalues lead.
#pragma once

#include <complex>
#include <vector>

namespace xb {

using cplx = std::complex<double>;

// Complex Schur form of the real m x m matrix A (row-major): Householder
// reduction to Hessenberg form, then shifted QR steps in complex arithmetic.
// T (upper triangular) and Z (unitary) are row-major m x m.  XB_ENOCONV if
// the QR iteration stalls.
int schur(int m, const double *A, std::vector<cplx> &T, std::vector<cplx> &Z);

// Eigenvalues on T's diagonal in wanted order (which = XB_EIG_LR: largest
// real part first; XB_EIG_LM: largest modulus first).  ord[t] = diagonal
// index of the t-th eigenvalue; kind[t] = 0 for a real eigenvalue, +1 / -1
// for the first (positive imaginary part) / second member of a conjugate
// pair, which are adjacent.  w[t] = the eigenvalue (imaginary part zeroed
// for real ones, exact conjugates for pairs).
void eig_order(int m, const std::vector<cplx> &T, int which, std::vector<int> &ord,
               std::vector<signed char> &kind, std::vector<cplx> &w);

// Unitary reordering: the eigenvalues at diagonal positions ord[0..k-1] move
// to positions 0..k-1 in that order (adjacent swaps); Z follows.
void schur_reorder(int m, std::vector<cplx> &T, std::vector<cplx> &Z, const std::vector<int> &ord,
                   int k);

// Unit eigenvector (in A's basis) of the eigenvalue at diagonal position i of
// T: back substitution in T, then y = Z s; phase chosen so that the largest
// entry is real and positive; real_ev zeroes the (rounding-level) imaginary part.
void schur_eigvec(int m, const std::vector<cplx> &T, const std::vector<cplx> &Z, int i,
                  bool real_ev, std::vector<cplx> &y);

// The number of leading wanted eigenvalues to keep, k0 moved by one (up if
// room remains below m, else down) when it would split a conjugate pair.
int keep_count(const std::vector<signed char> &kind, int k0, int m);

// Orthonormal REAL basis (m x k column-major in Q) of the span of Z's first k
// columns, which must be closed under conjugation: pivoted Gram-Schmidt
// (two passes) over the 2k columns Re Z, Im Z.  Returns the number of
// columns found (k unless the span is not conjugation-closed).
int real_basis(int m, const std::vector<cplx> &Z, int k, std::vector<double> &Q);

}  // namespace xb
