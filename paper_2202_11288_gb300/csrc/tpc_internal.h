// Internal declarations shared by the host setup (tpc_host.cpp) and the device code.
#pragma once

#include <string>
#include <vector>

#include "../../include/tpcamg.h"

namespace tpc {

// One level in generator-plus-Cross form (eq. (3.7)).
//   Toeplitz blocks A, B_bar, C_bar, D_bar (N x N) as generators t[d + N - 1] = T(i, j),
//   d = i - j in [-(N-1), N-1]; Cross vectors p (column), q (row), xi (column), zeta (row),
//   each N long, 0-based; o the middle diagonal entry.
struct LevelForm {
  int k = 0;
  long long N = 0;  // N_k = 2^k - 1
  std::vector<double> tA, tB, tC, tD;
  std::vector<double> p, q, xi, zeta;
  double o = 0.0;
  // Non-Toeplitz tridiagonal part (weakly singular model of section 2.1 only, else empty):
  // entries (i, i-1), (i, i), (i, i+1) of the concatenated 0-based index i < 2N + 1.
  std::vector<double> bl, bd, bu;
  bool has_band() const { return !bd.empty(); }
  double gen(const std::vector<double>& t, long long d) const { return t[d + N - 1]; }
};

struct HostHierarchy {
  int K = 0, kc = 0, r = 0;
  std::vector<LevelForm> lev;          // lev[0] = finest (K), lev.back() = coarsest (kc)
  std::vector<double> coarse_inv;      // n_kc x n_kc inverse of the coarsest matrix, row major
};

// Validate parameters and build the hierarchy on the host (FP64). Returns a TPC_* code and
// writes a message into err on failure.
int build_host_hierarchy(const tpc_params& p, double delta, double h, int levels,
                         HostHierarchy& out, std::string& err);

// Inverse of the coarsest level of the 2-D system, A (x) Q + Q (x) A - (A (x) A) / d with
// A the level's dense matrix and Q = tridiag(q1, q0, q1) (row-major, (2N+1)^2 square).
int coarse_inverse_2d(const LevelForm& Lc, double q0, double q1, double d,
                      std::vector<double>& inv);

// Export layout of one level (see tpc_export_level).
size_t export_count(long long N);
void export_level(const LevelForm& L, double* dst);

// exp(-2 pi i j / m) for j in [0, count), written as interleaved (re, im) pairs.
void twiddles(long long m, long long count, std::vector<double>& out);

// Polled solve with host buffers (tpc_api.cu), used by the request server (tpc_server.cu).
struct AsyncSolve;
int async_begin_host(tpc_handle* H, const double* b_host, double* x_host, double tol,
                     AsyncSolve** out);
int async_poll(AsyncSolve* a, int* done);
void async_result(const AsyncSolve* a, int* status, int* iters, double* relres);
void async_free(AsyncSolve* a);
size_t handle_device_bytes(const tpc_handle* H);
// The same for 2-D handles (tpc_2d.cuh).
struct AsyncSolve2;
int async2d_begin_host(tpc2d_handle* H, const double* b_host, double* x_host, double tol,
                       AsyncSolve2** out);
int async2d_poll(AsyncSolve2* a, int* done);
void async2d_result(const AsyncSolve2* a, int* status, int* iters, double* relres);
void async2d_free(AsyncSolve2* a);
size_t handle2d_device_bytes(const tpc2d_handle* H);

}  // namespace tpc
