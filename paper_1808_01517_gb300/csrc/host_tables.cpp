// Host FP64 table builder (see host_tables.h).
//
// Basis (Sec. 1 cites Descoteaux et al. 2007 for the SH representation): real,
// symmetric, even l only, j = l(l+1)/2 + m;  m < 0: sqrt2 * Nbar P_l^|m| cos(|m| phi),
// m = 0: Nbar P_l^0,  m > 0: sqrt2 * Nbar P_l^m sin(m phi), Condon-Shortley phase
// included.  Evaluated with the fully normalised associated-Legendre recurrence
// and a Chebyshev recurrence for cos(m phi), sin(m phi) from x/rho, y/rho.
//
// Pseudo-inverse (Sec. 2.2, lb_lambda): P = (B^T B + lambda L)^-1 B^T,
// L = diag(l^2 (l+1)^2), by a Cholesky factorisation of the normal matrix.
//
// LSC geometry (Sec. 2.3): origin + rings x sectors points, ring r at polar
// angle r * radius / rings, azimuth 2 pi q / sectors in the frame
// e1 = normalise(a - (a.g) g) (a = axis of smallest |g_k|, lowest k on ties),
// e2 = g x e1.  Collapse matrices M_{s,k} = P_out,s B^K_{s,k}.
#include "host_tables.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>

namespace delimit {

static const double kPi = 3.14159265358979323846;

int sh_ncoef(int order) {
  if (order < 0 || (order & 1)) return -1;
  return (order + 1) * (order + 2) / 2;
}

void sh_eval(int order, const double g[3], double* out) {
  const double r = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double x = g[2] / r;
  if (x > 1) x = 1;
  if (x < -1) x = -1;
  const double rho = std::sqrt(g[0] * g[0] + g[1] * g[1]);
  const double cp = rho > 0 ? g[0] / rho : 1.0, sp = rho > 0 ? g[1] / rho : 0.0;
  const double s = std::sqrt(std::max(0.0, (1 - x) * (1 + x)));
  const int L = order;
  // cos(m phi), sin(m phi) for m = 0..L
  std::vector<double> cm(L + 1), sm(L + 1);
  cm[0] = 1;
  sm[0] = 0;
  for (int m = 1; m <= L; ++m) {
    cm[m] = cm[m - 1] * cp - sm[m - 1] * sp;
    sm[m] = sm[m - 1] * cp + cm[m - 1] * sp;
  }
  // fully normalised Pbar_l^m(x) = sqrt((2l+1)/4pi (l-m)!/(l+m)!) P_l^m(x), CS phase included
  std::vector<double> pbar((L + 1) * (L + 1), 0.0);
  auto at = [&](int l, int m) -> double& { return pbar[l * (L + 1) + m]; };
  at(0, 0) = 1.0 / std::sqrt(4 * kPi);
  for (int m = 1; m <= L; ++m) at(m, m) = -std::sqrt((2.0 * m + 1) / (2.0 * m)) * s * at(m - 1, m - 1);
  for (int m = 0; m < L; ++m) at(m + 1, m) = std::sqrt(2.0 * m + 3) * x * at(m, m);
  for (int m = 0; m <= L; ++m)
    for (int l = m + 2; l <= L; ++l) {
      const double a = std::sqrt((4.0 * l * l - 1) / (double(l) * l - double(m) * m));
      const double b = std::sqrt((double(l - 1) * (l - 1) - double(m) * m) / (4.0 * (l - 1) * (l - 1) - 1));
      at(l, m) = a * (x * at(l - 1, m) - b * at(l - 2, m));
    }
  const double rt2 = std::sqrt(2.0);
  for (int l = 0; l <= L; l += 2) {
    const int base = l * (l + 1) / 2;
    out[base] = at(l, 0);
    for (int m = 1; m <= l; ++m) {
      out[base - m] = rt2 * at(l, m) * cm[m];
      out[base + m] = rt2 * at(l, m) * sm[m];
    }
  }
}

// Solves (B^T B + lambda L) P = B^T for P (N x m). Returns false if not positive definite.
static bool regularised_pinv(const std::vector<double>& B, int m, int N, int order, double lambda,
                             std::vector<double>& P) {
  std::vector<double> A(N * N, 0.0);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b <= a; ++b) {
      double acc = 0;
      for (int i = 0; i < m; ++i) acc += B[i * N + a] * B[i * N + b];
      A[a * N + b] = A[b * N + a] = acc;
    }
  int j = 0;
  for (int l = 0; l <= order; l += 2)
    for (int mm = -l; mm <= l; ++mm, ++j) A[j * N + j] += lambda * double(l) * (l + 1) * double(l) * (l + 1);
  double maxd = 0;
  for (int a = 0; a < N; ++a) maxd = std::max(maxd, std::fabs(A[a * N + a]));
  // Cholesky A = C C^T (lower C stored in A)
  for (int c = 0; c < N; ++c) {
    double d = A[c * N + c];
    for (int k = 0; k < c; ++k) d -= A[c * N + k] * A[c * N + k];
    if (!(d > 1e-12 * maxd)) return false;
    d = std::sqrt(d);
    A[c * N + c] = d;
    for (int r = c + 1; r < N; ++r) {
      double v = A[r * N + c];
      for (int k = 0; k < c; ++k) v -= A[r * N + k] * A[c * N + k];
      A[r * N + c] = v / d;
    }
  }
  P.assign(N * m, 0.0);
  std::vector<double> y(N);
  for (int col = 0; col < m; ++col) {
    for (int r = 0; r < N; ++r) {  // C y = b
      double v = B[col * N + r];
      for (int k = 0; k < r; ++k) v -= A[r * N + k] * y[k];
      y[r] = v / A[r * N + r];
    }
    for (int r = N - 1; r >= 0; --r) {  // C^T x = y
      double v = y[r];
      for (int k = r + 1; k < N; ++k) v -= A[k * N + r] * P[k * m + col];
      P[r * m + col] = v / A[r * N + r];
    }
  }
  return true;
}

int build_basis(const double* dirs, const double* bvals, int n, int order, double lambda, BasisHost& out,
                std::string& err, bool need_pinv) {
  char buf[256];
  const int N = sh_ncoef(order);
  if (N < 0 || order > 16) {
    err = "SH order must be even and in [0, 16]";
    return 1;
  }
  if (!dirs || !bvals || n <= 0) {
    err = "need at least one direction (non-null dirs and bvals)";
    return 1;
  }
  if (!(lambda >= 0) || !std::isfinite(lambda)) {
    err = "lambda must be finite and >= 0";
    return 1;
  }
  std::map<long long, std::vector<int>> groups;
  for (int i = 0; i < n; ++i) {
    const double* g = dirs + 3 * i;
    const double nr = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(std::fabs(nr - 1.0) <= 1e-6)) {
      std::snprintf(buf, sizeof buf, "direction %d has norm %.9g (need 1 +- 1e-6)", i, nr);
      err = buf;
      return 1;
    }
    const long long b = std::llround(bvals[i]);
    if (!(bvals[i] > 0) || b <= 0) {
      std::snprintf(buf, sizeof buf, "row %d has b = %g; remove b = 0 rows and normalise by b0 first", i,
                    bvals[i]);
      err = buf;
      return 1;
    }
    groups[b].push_back(i);
  }
  out = BasisHost();
  out.order = order;
  out.N = N;
  out.n_dirs = n;
  out.lambda = lambda;
  out.has_pinv = need_pinv;
  int off = 0;
  for (auto& kv : groups) {
    ShellHost sh;
    sh.bval = double(kv.first);
    sh.m = int(kv.second.size());
    sh.dir_off = off;
    sh.dir_index = kv.second;
    sh.dirs.resize(3 * sh.m);
    sh.B.resize(size_t(sh.m) * N);
    for (int i = 0; i < sh.m; ++i) {
      const double* g = dirs + 3 * kv.second[i];
      for (int k = 0; k < 3; ++k) sh.dirs[3 * i + k] = g[k];
      sh_eval(order, g, &sh.B[size_t(i) * N]);
    }
    if (!need_pinv) {
      sh.P.assign(size_t(N) * sh.m, 0.0);
    } else if (!regularised_pinv(sh.B, sh.m, N, order, lambda, sh.P)) {
      std::snprintf(buf, sizeof buf,
                    "shell b=%lld: normal matrix not positive definite (%d directions, %d coefficients, "
                    "lambda=%g)",
                    kv.first, sh.m, N, lambda);
      err = buf;
      return 2;
    }
    off += sh.m;
    out.shells.push_back(std::move(sh));
  }
  return 0;
}

// Resampling-free form for output shell s (tables already hold its kernel points):
// for every input shell s', the acquired neighbours j of each direction i
// (|g_i.g_j| >= cos(radius), ascending j), each oriented onto g_i's hemisphere and
// binned to the kernel point with the largest p_{i,k}.u (lowest k on ties); then
//   M_{s,s',k}[a][b] = sum_i P_out[a][i] * mean_{j in bin (i,k)} Y_b(g_j).
static void build_neighbour_form(const BasisHost& ob, int s, int order_in, int n_in, double cos_r, LscShellHost& L) {
  const ShellHost& sh = ob.shells[s];
  const int S = int(ob.shells.size()), m = sh.m, No = ob.N;
  const int K = int(L.kpts.size() / (size_t(m) * 3));
  L.M.assign(size_t(S) * K * No * n_in, 0.0);
  L.pair_indptr.assign(S, {});
  L.pair_indices.assign(S, {});
  L.pair_bins.assign(S, {});
  std::vector<double> mean(size_t(K) * n_in), y(n_in);
  std::vector<int> count(K);
  for (int p = 0; p < S; ++p) {
    const ShellHost& sp = ob.shells[p];
    auto& indptr = L.pair_indptr[p];
    auto& indices = L.pair_indices[p];
    auto& bins = L.pair_bins[p];
    indptr.assign(1, 0);
    double* Mp = &L.M[size_t(p) * K * No * n_in];
    for (int i = 0; i < m; ++i) {
      const double* gi = &sh.dirs[3 * i];
      const double* kp = &L.kpts[size_t(i) * K * 3];
      std::fill(mean.begin(), mean.end(), 0.0);
      std::fill(count.begin(), count.end(), 0);
      for (int j = 0; j < sp.m; ++j) {
        const double* gj = &sp.dirs[3 * j];
        const double d = gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
        if (!(std::fabs(d) >= cos_r)) continue;
        const double sg = d >= 0.0 ? 1.0 : -1.0;
        const double u[3] = {sg * gj[0], sg * gj[1], sg * gj[2]};
        int best = 0;
        double best_c = kp[0] * u[0] + kp[1] * u[1] + kp[2] * u[2];
        for (int k = 1; k < K; ++k) {
          const double c = kp[3 * k] * u[0] + kp[3 * k + 1] * u[1] + kp[3 * k + 2] * u[2];
          if (c > best_c) best_c = c, best = k;
        }
        indices.push_back(j);
        bins.push_back(best);
        sh_eval(order_in, gj, y.data());  // even order: Y(-g) = Y(g)
        for (int b = 0; b < n_in; ++b) mean[size_t(best) * n_in + b] += y[b];
        ++count[best];
      }
      indptr.push_back((long long)indices.size());
      for (int k = 0; k < K; ++k) {
        if (!count[k]) continue;
        const double inv = 1.0 / count[k];
        const double* mk = &mean[size_t(k) * n_in];
        for (int a = 0; a < No; ++a) {
          const double pa = sh.P[size_t(a) * m + i] * inv;
          double* row = &Mp[(size_t(k) * No + a) * n_in];
          for (int b = 0; b < n_in; ++b) row[b] += pa * mk[b];
        }
      }
    }
  }
}

int build_lsc(const BasisHost& ob, int order_in, int shells_in, double radius, int rings, int sectors, int window,
              bool neighbours, LscHost& out, std::string& err) {
  const int n_in = sh_ncoef(order_in);
  if (n_in < 0 || order_in > 16) {
    err = "order_in must be even and in [0, 16]";
    return 1;
  }
  if (!(radius > 0) || radius > kPi / 2 || rings < 1 || sectors < 1 || rings * sectors > 1024) {
    err = "need 0 < radius <= pi/2, rings >= 1, sectors >= 1, rings*sectors <= 1024";
    return 1;
  }
  const int s_out = int(ob.shells.size());
  if (shells_in < 1 || shells_in > 64) {
    err = "shells_in must be in [1, 64]";
    return 1;
  }
  if (window != -1 && window != 0 && window != 1) {
    err = "window must be DELIMIT_WINDOW_SAME, _ADJACENT or _ALL";
    return 1;
  }
  if (window != -1 && shells_in != s_out) {
    err = "same/adjacent windows need shells_in equal to the output basis' shell count";
    return 1;
  }
  if (neighbours && shells_in != s_out) {
    err = "the resampling-free LSC samples input shell s' on the table's shell s': shells_in must equal its shell count";
    return 1;
  }
  if (neighbours && double(s_out) * s_out * (1 + rings * sectors) * ob.N * n_in * 8.0 > double(1 << 28)) {
    err = "resampling-free LSC: the per-shell-pair collapse matrices would exceed 256 MiB";
    return 1;
  }
  out = LscHost();
  out.neighbours = neighbours;
  out.order_in = order_in;
  out.n_in = n_in;
  out.n_out = ob.N;
  out.s_in = shells_in;
  out.s_out = s_out;
  out.rings = rings;
  out.sectors = sectors;
  out.K = 1 + rings * sectors;
  out.radius = radius;
  out.window = window;
  const int K = out.K, No = ob.N;
  const double cos_r = std::cos(radius);
  std::vector<double> bk(n_in);
  for (int s = 0; s < s_out; ++s) {
    const ShellHost& sh = ob.shells[s];
    LscShellHost L;
    const int m = sh.m;
    L.kpts.resize(size_t(m) * K * 3);
    // B^K: basis of order_in at every kernel point, [m][K][n_in]
    std::vector<double> BK(size_t(m) * K * n_in);
    for (int i = 0; i < m; ++i) {
      const double* g = &sh.dirs[3 * i];
      int ax = 0;
      for (int k = 1; k < 3; ++k)
        if (std::fabs(g[k]) < std::fabs(g[ax])) ax = k;
      double e1[3] = {0, 0, 0};
      e1[ax] = 1.0;
      const double ag = g[ax];
      for (int k = 0; k < 3; ++k) e1[k] -= ag * g[k];
      const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
      for (int k = 0; k < 3; ++k) e1[k] /= n1;
      const double e2[3] = {g[1] * e1[2] - g[2] * e1[1], g[2] * e1[0] - g[0] * e1[2], g[0] * e1[1] - g[1] * e1[0]};
      for (int k = 0; k < K; ++k) {
        double p[3];
        if (k == 0) {
          p[0] = g[0], p[1] = g[1], p[2] = g[2];
        } else {
          const int r = (k - 1) / sectors + 1, q = (k - 1) % sectors;
          const double th = r * radius / rings, ph = 2.0 * kPi * q / sectors;
          const double ct = std::cos(th), st = std::sin(th), cph = std::cos(ph), sph = std::sin(ph);
          for (int d = 0; d < 3; ++d) p[d] = ct * g[d] + st * (cph * e1[d] + sph * e2[d]);
        }
        for (int d = 0; d < 3; ++d) L.kpts[(size_t(i) * K + k) * 3 + d] = p[d];
        sh_eval(order_in, p, &BK[(size_t(i) * K + k) * n_in]);
      }
    }
    // M_{s,k}[a][b] = sum_i P_out[a][i] * BK[i][k][b]
    L.M.assign(size_t(K) * No * n_in, 0.0);
    for (int k = 0; !neighbours && k < K; ++k)
      for (int a = 0; a < No; ++a) {
        double* row = &L.M[(size_t(k) * No + a) * n_in];
        for (int i = 0; i < m; ++i) {
          const double pa = sh.P[size_t(a) * m + i];
          const double* bkr = &BK[(size_t(i) * K + k) * n_in];
          for (int b = 0; b < n_in; ++b) row[b] += pa * bkr[b];
        }
      }
    L.q.assign(No, 0.0);
    for (int a = 0; a < No; ++a)
      for (int i = 0; i < m; ++i) L.q[a] += sh.P[size_t(a) * m + i];
    // neighbour table T3 (antipodal-aware, ascending, equality counts as inside)
    L.nb_indptr.assign(1, 0);
    for (int i = 0; i < m; ++i) {
      const double* gi = &sh.dirs[3 * i];
      for (int j = 0; j < m; ++j) {
        const double* gj = &sh.dirs[3 * j];
        const double d = gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
        if (std::fabs(d) >= cos_r) L.nb_indices.push_back(j);
      }
      L.nb_indptr.push_back((long long)L.nb_indices.size());
    }
    // window table T2
    L.window.assign(shells_in, 0);
    for (int p = 0; p < shells_in; ++p)
      L.window[p] = (window == -1) ? 1 : (window == 0 ? (p == s) : (std::abs(p - s) <= 1));
    if (neighbours) build_neighbour_form(ob, s, order_in, n_in, cos_r, L);
    out.shells.push_back(std::move(L));
  }
  return 0;
}

}  // namespace delimit
