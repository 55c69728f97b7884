// Host driver of the partitioned band solve's per-thread routines
// (band_spike.cuh), for the CPU tests: every thread index of every kernel
// launch is run in turn, in launch order, with the same arguments the GPU
// launches pass.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "band_spike.cuh"

using namespace asv::spk;

namespace {

// The warp kernels' phase runner on the host: the 32 lanes of a phase in
// turn, in increasing or (to expose any dependence between the lanes of one
// phase) decreasing order.
bool g_reverse = false;
auto lanes = [](auto&& f) {
  for (int k = 0; k < 32; ++k) f(g_reverse ? 31 - k : k);
};

void solve_sys(const Ctx& c, bool tr, const std::vector<double>& M, const std::vector<int>& piv, double* x,
               bool warp, bool win) {
  const int64_t q = q_of(c);
  std::vector<double> G((size_t)c.n), Y((size_t)(c.P * (q > 0 ? q : 1)));
  double red[32];
  for (int64_t b = 0; b < c.P; ++b)
    if (warp) wsolve_step1(c, tr, b, x, G.data(), red, lanes);
    else solve_step1(c, tr, b, x, G.data());
  if (q > 0)
    for (int64_t b = 0; b + 1 < c.P; ++b)
      if (win) wsolve_step2(c, tr, b, G.data(), M.data(), piv.data(), Y.data(), lanes);
      else solve_step2(c, tr, b, G.data(), M.data(), piv.data(), Y.data());
  for (int64_t b = 0; b < c.P; ++b)
    if (warp) wsolve_step3(c, tr, b, Y.data(), x, red, lanes);
    else solve_step3(c, tr, b, Y.data(), x);
}

}  // namespace

// AB: A in band storage, A(i,j) at AB[ku + i - j + j*ldab].  Solves A x = b
// into x and A^T xt = b into xt (b: n values).  far[0], far[1]: the largest
// far-tip entry for A and for A^T; dom[0], dom[1]: dominance by rows / by
// columns.  warp: the one-warp-per-block factorisation and block solves
// (lanes run phase by phase; 2: lanes in decreasing order) instead of one
// thread per block; 3 (4: lanes in decreasing order): the routines of the
// route for bands up to 32 wide -- window spike columns, the one-phase-per-
// column block factorisation, the boundary systems and their solves by one
// warp (the block solves, whose GPU form uses warp shuffles, as in mode 1).
// Returns 0,
// -1 - b if block b has a zero pivot, -1000 - b if boundary system b is
// singular.
extern "C" int spike_host_solve(const double* AB, int64_t ldab, int kl, int ku, int64_t n, int64_t m,
                                const double* bvec, double* x, double* xt, double* far, int* dom, int warp) {
  g_reverse = warp == 2 || warp == 4;
  const bool win = warp >= 3;
  const int64_t ldf = 2 * (int64_t)kl + ku + 1, kv = (int64_t)kl + ku;
  std::vector<double> F((size_t)(ldf * n), 0.0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = j - ku; i <= j + kl; ++i)
      if (i >= 0 && i < n) F[(size_t)(kv + i - j + j * ldf)] = AB[(size_t)(ku + i - j + j * ldab)];
  Ctx c{F.data(), ldf, n, kl, ku, m, n / m};
  dom[0] = dom[1] = 1;
  for (int64_t i = 0; i < n; ++i) {
    int r, cc;
    dominance(c, i, &r, &cc);
    dom[0] &= r;
    dom[1] &= cc;
  }
  std::vector<double> rd((size_t)n);
  for (int64_t b = 0; b < c.P; ++b)
    if (win ? wfactor_block_step(c, b, rd.data(), lanes) : warp ? wfactor_block(c, b, lanes) : factor_block(c, b))
      return (int)(-1 - b);
  if (!win)
    for (int64_t i = 0; i < n; ++i) rd[(size_t)i] = 1.0 / F[(size_t)(kv + i * ldf)];
  const int64_t q = q_of(c);
  std::vector<double> scr((size_t)(n * (q > 0 ? q : 1)));
  std::vector<double> M[2];
  std::vector<int> piv[2];
  for (int tr = 0; tr < 2; ++tr) {
    M[tr].assign((size_t)(c.P * q * q + 1), 0.0);
    piv[tr].assign((size_t)(c.P * q + 1), 0);
    unsigned long long fb = 0;
    for (int64_t t = 0; t < c.P * q; ++t)
      if (win) spike_column_win(c, tr != 0, t, scr.data(), M[tr].data(), &fb, rd.data());
      else spike_column(c, tr != 0, t, scr.data(), M[tr].data(), &fb);
    memcpy(&far[tr], &fb, sizeof(double));
    double rv[33];
    int ri[33];
    for (int64_t b = 0; b + 1 < c.P; ++b)
      if (q > 0 && (win ? wfactor_boundary(c, b, M[tr].data(), piv[tr].data(), rv, ri, lanes)
                        : factor_boundary(c, b, M[tr].data(), piv[tr].data())))
        return (int)(-1000 - b);
  }
  memcpy(x, bvec, sizeof(double) * (size_t)n);
  memcpy(xt, bvec, sizeof(double) * (size_t)n);
  solve_sys(c, false, M[0], piv[0], x, warp != 0, win);
  solve_sys(c, true, M[1], piv[1], xt, warp != 0, win);
  return 0;
}
