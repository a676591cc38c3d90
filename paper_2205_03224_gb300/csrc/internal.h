// Internal types of the GB300 GeMSLR library (host side).
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "gemslr.h"

namespace gemslr {

// Host CSR (0-based, ascending columns).
struct Csr {
    int64_t nrows = 0, ncols = 0;
    std::vector<int64_t> rp{0};
    std::vector<int32_t> ci;
    std::vector<double> v;
    std::vector<double> vi;          // imaginary parts (complex factors); empty: real
    int64_t nnz() const { return (int64_t)ci.size(); }
};

// Exceptions used inside the library; converted to a status at the ABI.
struct Error {
    gemslr_status st;
    std::string msg;
};
[[noreturn]] void fail(gemslr_status st, const std::string &msg);

// u in [0, 1) from splitmix64(seed): the first `count` outputs' top 53 bits
// (the seeded start vectors and random blocks of the set-up; setup.cpp).
std::vector<double> splitmix_uniform01(uint64_t seed, int64_t count);

// ---- sparse utilities (setup.cpp) ----------------------------------------
Csr csr_from_abi(const gemslr_csr *A);
Csr csr_from_mat(const gemslr_mat &m);
Csr permute_sym(const Csr &A, const std::vector<int32_t> &perm);
Csr submatrix(const Csr &A, int64_t r0, int64_t r1, int64_t c0, int64_t c1);
Csr block_diag_part(const Csr &A, const std::vector<int64_t> &bp);   // keep in-block entries
bool blocks_coupled(const Csr &A, const std::vector<int64_t> &bp);   // any off-block entry

// Incomplete LU of one block (local numbering).  L strictly lower, U upper
// with the diagonal first in each row.  Returns the number of clamped pivots.
int64_t factor_ilu0(const Csr &B, Csr &L, Csr &U);
int64_t factor_ilut(const Csr &B, double tau, int lfil, Csr &L, Csr &U);
void append_block(Csr &dst, const Csr &blk, int64_t off);            // block-diagonal assembly

// Level sets (wavefronts) of a triangular factor restricted to one block.
// level[i] = 1 + max level of its dependencies (L: columns < i, U: > i).
std::vector<int32_t> wavefronts_lower(const Csr &L, int64_t r0, int64_t r1);
std::vector<int32_t> wavefronts_upper(const Csr &U, int64_t r0, int64_t r1);

// ---- partitioner (partition.cpp) ------------------------------------------
void local_order(const int32_t *coords, int64_t n, const std::vector<int64_t> &level_ptr,
                 const std::vector<int32_t> &nblk, const std::vector<int64_t> &block_ptr, int first,
                 std::vector<int32_t> &perm);
void partition_geometric(const Csr &A, const int32_t *coords, int nlev, int p, int p_last,
                         std::vector<int32_t> &perm, std::vector<int64_t> &level_ptr,
                         std::vector<int32_t> &nblk, std::vector<int64_t> &block_ptr);

// ---- dense Schur machinery (schur.cpp) ------------------------------------
// Given a real m x m matrix Hm (column-major), select the k wanted Ritz values
// by |theta/(1-theta)| (pairs kept whole) and return an orthonormal real
// basis Q (m x keff, column-major) of their invariant subspace and
// Tk = Q^T Hm Q (keff x keff).  theta receives the wanted values (re, im).
int schur_wanted(const std::vector<double> &Hm, int m, int k, std::vector<double> &Q,
                 std::vector<double> &Tk, std::vector<double> &theta_re,
                 std::vector<double> &theta_im);
// H = (I - Tk)^{-1} - I (k x k, column-major), partial pivoting LU.
std::vector<double> correction_matrix(const std::vector<double> &Tk, int k);
// Complex counterparts (complex-shifted hierarchy, Sec. 5.2.3): complex Schur
// form of a general complex m x m Hm, the k wanted values (same ranking, no
// pairs) leading; Q (m x k) and the upper triangular Tk (k x k), column-major.
int schur_wanted_z(const std::vector<std::complex<double>> &Hm, int m, int k,
                   std::vector<std::complex<double>> &Q, std::vector<std::complex<double>> &Tk,
                   std::vector<std::complex<double>> &theta);
std::vector<std::complex<double>> correction_matrix_z(const std::vector<std::complex<double>> &Tk, int k);

// ---- host description of the hierarchy -------------------------------------
struct HostLevel {
    int64_t s = 0, e = 0;            // level rows [s, e) in the multilevel order
    std::vector<int64_t> bp;         // block offsets, level-local, nblk+1
    Csr L, U;                        // level-local, block diagonal
    Csr E;                           // (n - e) x (e - s)
    Csr F;                           // (e - s) x (n - e)
    int k = 0;                       // rank (effective, pairs kept whole)
    int rank_req = 0;
    std::vector<double> W;           // (n - e) x k, column-major
    std::vector<double> H;           // k x k, column-major
    std::vector<double> Wi, Hi;      // imaginary parts of W and H (complex hierarchy); empty: real
};

struct Hierarchy {
    int64_t n = 0;
    int nlev = 0;
    std::vector<int32_t> perm;
    std::vector<int64_t> level_ptr;
    Csr Ahat;                        // P^T A P
    std::vector<HostLevel> lev;      // nlev - 1 Schur levels
    HostLevel last;                  // s, e = n, bp, L, U
    int64_t nclamp = 0;
    // complex diagonal shift of the factored blocks (Sec. 5.2.3): B + i alpha I;
    // with cplx the factors, W and H carry imaginary parts and M^{-1} is complex
    double alpha = 0.0;
    bool cplx = false;
};

// ILU(0) of the diagonal blocks of a level matrix on the current device (ilu_device.cu).
void factor_level_ilu0_device(const Csr &B, const std::vector<int64_t> &bp, Csr &L, Csr &U, int64_t &clamped);
// ILUT(tau, lfil) of the diagonal blocks of a level matrix on the current device
// (one warp per block, rows in order; bit-identical to factor_ilut; 0 <= lfil <= 64).
// false: a row was too wide for the kernel and nothing was written.
bool factor_level_ilut_device(const Csr &B, const std::vector<int64_t> &bp, double tau, int lfil, Csr &L, Csr &U,
                              int64_t &clamped);

// Build the hierarchy without the low-rank terms (permute, slice, factor).
void build_levels(const Csr &A, const gemslr_partition *part, const gemslr_options *opt,
                  Hierarchy &h);

}  // namespace gemslr
