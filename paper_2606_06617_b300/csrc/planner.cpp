// Host planner for PSWF-LR: see planner.hpp.  Plain C++17, FP64.
#include "planner.hpp"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>

#include "pswf_lr.h"

namespace pswf {

namespace {
constexpr double kPi = 3.14159265358979323846;

// P_n^{(m)}(x) for n <= nmax, m <= mmax (unnormalised Legendre), via
// (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1} and
// P^{(m)}_{n+1} = P^{(m)}_{n-1} + (2n+1) P^{(m-1)}_n.
void legendre_table(double x, int nmax, int mmax, std::vector<double>& T) {
  T.assign(size_t(mmax + 1) * (nmax + 1), 0.0);
  auto at = [&](int m, int n) -> double& { return T[size_t(m) * (nmax + 1) + n]; };
  at(0, 0) = 1.0;
  if (nmax >= 1) at(0, 1) = x;
  for (int n = 1; n < nmax; ++n) at(0, n + 1) = ((2.0 * n + 1.0) * x * at(0, n) - n * at(0, n - 1)) / (n + 1.0);
  for (int m = 1; m <= mmax; ++m) {
    if (nmax >= 1) at(m, 1) = (m == 1) ? 1.0 : 0.0;
    for (int n = 1; n < nmax; ++n) at(m, n + 1) = at(m, n - 1) + (2.0 * n + 1.0) * at(m - 1, n);
  }
}

// Chebyshev interpolation of f on [-1, 1] at n nodes; returns coefficients.
std::vector<double> cheb_fit(const std::function<double(double)>& f, int n) {
  std::vector<double> fx(n), a(n, 0.0);
  for (int k = 0; k < n; ++k) fx[k] = f(std::cos(kPi * (k + 0.5) / n));
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += fx[k] * std::cos(kPi * j * (k + 0.5) / n);
    a[j] = 2.0 * s / n;
  }
  a[0] *= 0.5;
  return a;
}

// Chebyshev coefficients a[0..deg] -> monomial coefficients in s.
std::vector<double> cheb_to_monomial(const std::vector<double>& a, int deg) {
  std::vector<double> out(deg + 1, 0.0);
  std::vector<double> tprev(deg + 1, 0.0), tcur(deg + 1, 0.0), tnext(deg + 1, 0.0);
  tprev[0] = 1.0;               // T_0
  if (deg >= 1) tcur[1] = 1.0;  // T_1
  for (int i = 0; i <= deg; ++i) out[i] += a[0] * tprev[i];
  if (deg >= 1)
    for (int i = 0; i <= deg; ++i) out[i] += a[1] * tcur[i];
  for (int j = 2; j <= deg; ++j) {
    std::fill(tnext.begin(), tnext.end(), 0.0);
    for (int i = 0; i < deg; ++i) tnext[i + 1] += 2.0 * tcur[i];
    for (int i = 0; i <= deg; ++i) tnext[i] -= tprev[i];
    for (int i = 0; i <= deg; ++i) out[i] += a[j] * tnext[i];
    tprev.swap(tcur);
    tcur.swap(tnext);
  }
  return out;
}

// Degree kept by the paper's filter (drop trailing |a_n| <= 0.01 eps max|a|)
// over a family of expansions, max|a| taken over the whole family so that
// pieces where the function is tiny do not chase round-off.
int family_degree(const std::vector<std::vector<double>>& fam, double eps) {
  double amax = 0.0;
  for (const auto& a : fam)
    for (double v : a) amax = std::max(amax, std::fabs(v));
  int d = 1;
  for (const auto& a : fam)
    for (int j = 0; j < int(a.size()); ++j)
      if (std::fabs(a[j]) > 0.01 * eps * amax) d = std::max(d, j);
  return d;
}

int fail(Plan& plan, int code, const char* msg) {
  plan.error = msg;
  return code;
}
}  // namespace

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

int64_t next_fft_size(int64_t n) {
  if (n < 1) n = 1;
  for (int64_t m = n;; ++m) {
    int64_t r = m;
    for (int f : {2, 3, 5, 7})
      while (r % f == 0) r /= f;
    if (r == 1) return m;
  }
}

Prolate::Prolate(double c_) : c(c_) {
  // Even Legendre coefficients only (psi_0 is even).
  const int N = std::max(30, int(1.2 * c) + 30);
  auto alpha = [](int n) -> double {
    if (n < 0) return 0.0;
    return (n + 1.0) / std::sqrt((2.0 * n + 1.0) * (2.0 * n + 3.0));
  };
  // Prolate operator -(d/dx)(1-x^2)(d/dx) + c^2 x^2 in the basis Pbar_{2k}:
  // x Pbar_n = alpha_n Pbar_{n+1} + alpha_{n-1} Pbar_{n-1}, so the matrix has
  // diagonal n(n+1) + c^2 (alpha_n^2 + alpha_{n-1}^2) and off-diagonal
  // (n, n+2) entries c^2 alpha_n alpha_{n+1}.
  std::vector<double> dg(N), of(N > 1 ? N - 1 : 1, 0.0);
  for (int k = 0; k < N; ++k) {
    const int n = 2 * k;
    dg[k] = n * (n + 1.0) + c * c * (alpha(n) * alpha(n) + alpha(n - 1) * alpha(n - 1));
    if (k + 1 < N) of[k] = c * c * alpha(n) * alpha(n + 1);
  }
  // The matrix is symmetric tridiagonal: smallest eigenvalue by Sturm-count
  // bisection, its eigenvector by inverse iteration (Thomas solves).
  auto below = [&](double x) {   // eigenvalues < x
    int cnt = 0;
    double q = dg[0] - x;
    if (q < 0) ++cnt;
    for (int k = 1; k < N; ++k) {
      const double qq = (q != 0.0) ? q : 1e-300;
      q = dg[k] - x - of[k - 1] * of[k - 1] / qq;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  double lo = dg[0], hi = dg[0];
  for (int k = 0; k < N; ++k) {
    const double r = (k > 0 ? std::fabs(of[k - 1]) : 0.0) + (k + 1 < N ? std::fabs(of[k]) : 0.0);
    lo = std::min(lo, dg[k] - r);
    hi = std::max(hi, dg[k] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= 1)
      hi = mid;
    else
      lo = mid;
  }
  chi = 0.5 * (lo + hi);
  std::vector<double> v(N, 1.0), w(N), cp(N), dp(N);
  const double shift = chi - 1e-10 * std::max(1.0, std::fabs(chi));
  for (int it = 0; it < 4; ++it) {
    // solve (T - shift I) w = v
    double den = dg[0] - shift;
    cp[0] = (N > 1 ? of[0] : 0.0) / den;
    dp[0] = v[0] / den;
    for (int k = 1; k < N; ++k) {
      den = dg[k] - shift - of[k - 1] * cp[k - 1];
      cp[k] = (k + 1 < N ? of[k] : 0.0) / den;
      dp[k] = (v[k] - of[k - 1] * dp[k - 1]) / den;
    }
    w[N - 1] = dp[N - 1];
    for (int k = N - 2; k >= 0; --k) w[k] = dp[k] - cp[k] * w[k + 1];
    double nrm = 0.0;
    for (int k = 0; k < N; ++k) nrm += w[k] * w[k];
    nrm = std::sqrt(nrm);
    for (int k = 0; k < N; ++k) v[k] = w[k] / nrm;
  }
  beta = v;
  double s = 0.0;
  {
    std::vector<double> T;
    legendre_table(0.0, 2 * N, 0, T);
    for (int k = 0; k < N; ++k) s += beta[k] * std::sqrt(2 * k + 0.5) * T[2 * k];
  }
  for (double& b : beta) b /= s;  // psi(0) = 1
  bs.resize(N);
  for (int k = 0; k < N; ++k) bs[k] = beta[k] * std::sqrt(2 * k + 0.5);
  // lambda_0 = int_{-1}^{1} psi = beta_0 int Pbar_0 = beta_0 sqrt(2)
  lambda0 = beta[0] * std::sqrt(2.0);
  C0 = 0.5 * lambda0;
}

double Prolate::eval(double x, int m) const {
  const int N = int(beta.size());
  if (m == 0) {
    // sum_k bs_k P_{2k}(x) along the three-term recurrence (no table)
    double p0 = 1.0, p1 = x, sum = bs[0];
    for (int n = 1; n + 1 <= 2 * N - 2; ++n) {
      const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
      p0 = p1;
      p1 = p2;
      if (((n + 1) & 1) == 0) sum += bs[(n + 1) / 2] * p1;
    }
    return sum;
  }
  std::vector<double> T;
  legendre_table(x, 2 * N, m, T);
  const double* Pm = T.data() + size_t(m) * (2 * N + 1);
  double s = 0.0;
  for (int k = 0; k < N; ++k) s += beta[k] * std::sqrt(2 * k + 0.5) * Pm[2 * k];
  return s;
}

double Prolate::integral(double a, double b, int power) const {
  static thread_local std::vector<double> gx, gw;
  if (gx.size() != 64) gauss_legendre(64, gx, gw);
  const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
  double s = 0.0;
  for (int i = 0; i < 64; ++i) {
    const double t = mid + half * gx[i];
    s += gw[i] * std::pow(t, power) * eval(t);
  }
  return s * half;
}

// Smooth parts of Eq. (PhiH) after the substitution x = c s, with psi_0(x/c) taken as zero for x > c
// (psi_0(x/c) = 0 for x > c), u = k r_c / c, with
//   I(u) = int_0^u psi, J1(u) = int_u^1 s psi, J3(u) = int_u^1 s^3 psi,
//   H(u) = int_u^1 (psi(s) - 1) / s ds:
//   p=1: Phi = 4 pi / k^2           * psi(u)
//   p=2: Phi = 2 pi^2 / k            * (1 - I/C0)
//   p=3: Phi = 4 pi                  * (-log u + H)
//   p=4: Phi = pi^2 c / r_c          * (J1/C0 - u (1 - I/C0))
//   p=5: Phi = -2 pi c^2 / (3 r_c^2) * (u^2 (-log u + H) - J1)
//   p=6: Phi = pi^2 c^3/(12 r_c^3)   * (u^3 (1 - I/C0) - 3 u^2 J1/(2 C0) + J3/(2 C0))
// This function returns the log-free part (H in place of -log u + H).
double mult_smooth(const Prolate& ps, int p, double u) {
  const double C0 = ps.C0;
  auto I = [&]() { return u > 0 ? ps.integral(0.0, u, 0) : 0.0; };
  auto J1 = [&]() { return u < 1 ? ps.integral(u, 1.0, 1) : 0.0; };
  auto J3 = [&]() { return u < 1 ? ps.integral(u, 1.0, 3) : 0.0; };
  auto H = [&]() {
    if (u >= 1) return 0.0;
    static thread_local std::vector<double> gx, gw;
    if (gx.size() != 64) gauss_legendre(64, gx, gw);
    const double half = 0.5 * (1.0 - u), mid = 0.5 * (1.0 + u);
    double s = 0.0;
    for (int i = 0; i < 64; ++i) {
      const double t = mid + half * gx[i];
      s += gw[i] * (ps.eval(t) - 1.0) / t;
    }
    return s * half;
  };
  switch (p) {
    case 1: return ps.eval(u);
    case 2: return 1.0 - I() / C0;
    case 3: return H();
    case 4: return J1() / C0 - u * (1.0 - I() / C0);
    case 5: return u * u * H() - J1();
    case 6: return u * u * u * (1.0 - I() / C0) - 1.5 * u * u * J1() / C0 + 0.5 * J3() / C0;
    default: return 0.0;
  }
}

namespace {

// Chebyshev fits of the multiplier smooth part S_p on the kMultSeg pieces of
// [0, 1]: they depend only on (c, p, precision), so plans share them.
struct MultFit {
  int deg = 1;
  std::vector<std::vector<double>> cheb;   // [kMultSeg]
};

const MultFit& mult_fit(const Prolate& moll, int p, double eps_poly) {
  static std::mutex mu;
  static std::map<std::tuple<double, int, double>, MultFit> cache;
  const auto key = std::make_tuple(moll.c, p, eps_poly);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  MultFit f;
  const int nfit = 33;
  f.cheb.resize(kMultSeg);
  for (int i = 0; i < kMultSeg; ++i) {
    const double a = double(i) / kMultSeg, b = double(i + 1) / kMultSeg;
    f.cheb[i] = cheb_fit([&](double sv) { return mult_smooth(moll, p, a + (b - a) * 0.5 * (sv + 1.0)); }, nfit);
  }
  f.deg = family_degree(f.cheb, eps_poly);
  std::lock_guard<std::mutex> lk(mu);
  return cache.emplace(key, std::move(f)).first->second;
}

// Real-space mollifier G_p(x), x = r / r_c in [0, 1] (Eq. G1, G6, G of the
// Methods; G_p taken as 1 beyond r_c), with I(x) = int_0^x psi.
double real_mollifier(const Prolate& ps, int p, double x) {
  const double C0 = ps.C0;
  const double I = x > 0 ? ps.integral(0.0, x, 0) : 0.0;
  switch (p) {
    case 1: return I / C0;
    case 2: return 1.0 - ps.eval(x);
    case 3: return (I - x * ps.eval(x)) / C0;
    case 4: return 1.0 - ps.eval(x) + 0.5 * x * ps.eval(x, 1);
    case 5: return (I - x * ps.eval(x) + x * x / 3.0 * ps.eval(x, 1)) / C0;
    case 6: return 1.0 - ps.eval(x) + 0.625 * x * ps.eval(x, 1) - 0.125 * x * x * ps.eval(x, 2);
    default: return 1.0;
  }
}

// Chebyshev fits of G_p on the kMultSeg pieces of [0, 1], shared like the
// multiplier fits.
const MultFit& real_fit(const Prolate& moll, int p, double eps_poly) {
  static std::mutex mu;
  static std::map<std::tuple<double, int, double>, MultFit> cache;
  const auto key = std::make_tuple(moll.c, p, eps_poly);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  MultFit f;
  const int nfit = 33;
  f.cheb.resize(kMultSeg);
  for (int i = 0; i < kMultSeg; ++i) {
    const double a = double(i) / kMultSeg, b = double(i + 1) / kMultSeg;
    f.cheb[i] = cheb_fit([&](double sv) { return real_mollifier(moll, p, a + (b - a) * 0.5 * (sv + 1.0)); }, nfit);
  }
  f.deg = family_degree(f.cheb, eps_poly);
  std::lock_guard<std::mutex> lk(mu);
  return cache.emplace(key, std::move(f)).first->second;
}

// Everything that depends on the grid spacing at box_max and on the set of
// exponents, but not on a particular structure.
int plan_core(const double box_max[3], int K, const int* pset, int npset, const Options& opt, Plan& plan) {
  plan.opt = opt;
  for (int d = 0; d < 3; ++d) {
    if (!(box_max[d] > 0.0) || !std::isfinite(box_max[d]))
      return fail(plan, PSWF_EINVAL, "box edges must be positive and finite");
    plan.box_max[d] = box_max[d];
    plan.box[d] = box_max[d];
  }
  if (K < 1 || K > kMaxK) return fail(plan, PSWF_EINVAL, "number of channels must be in 1..64");
  plan.K = K;
  bool use_p[7] = {false, false, false, false, false, false, false};
  for (int k = 0; k < npset; ++k) {
    if (pset[k] < 1 || pset[k] > 6) return fail(plan, PSWF_EINVAL, "channel exponent p must be in 1..6");
    use_p[pset[k]] = true;
  }
  if (!(opt.r_c > 0.0) || !std::isfinite(opt.r_c)) return fail(plan, PSWF_EINVAL, "r_c must be positive");
  if (!(opt.tol > 0.0 && opt.tol < 1.0)) return fail(plan, PSWF_EINVAL, "tol must be in (0, 1)");
  if (opt.precision != 0 && opt.precision != 1) return fail(plan, PSWF_EINVAL, "precision must be 0 (fp32) or 1 (fp64)");
  plan.tol = opt.tol;
  plan.r_c = opt.r_c;
  // ---- Parameter selection: eps_band = eps_grid = eps_spread = tol / 3 ----
  plan.c = opt.c > 0 ? opt.c : std::log(3.0 / opt.tol);
  if (plan.c > 60.0) return fail(plan, PSWF_EINVAL, "c must be <= 60");
  plan.k_c = plan.c / plan.r_c;
  const double eta_t = opt.eta > 0 ? opt.eta : 0.5;
  if (eta_t >= 1.0) return fail(plan, PSWF_EINVAL, "eta must be in (0, 1)");
  for (int d = 0; d < 3; ++d) {
    const int64_t M = opt.grid[d] > 0 ? opt.grid[d]
                                      : next_fft_size(int64_t(std::ceil(box_max[d] * plan.k_c / (eta_t * kPi))));
    if (M < 2 || M > 4096) return fail(plan, PSWF_EINVAL, "grid size per dimension must be in 2..4096");
    plan.M[d] = int(M);
    plan.h[d] = box_max[d] / double(M);
  }
  plan.eta = 0.0;
  for (int d = 0; d < 3; ++d) plan.eta = std::max(plan.eta, plan.h[d] * plan.k_c / kPi);
  if (plan.eta >= 1.0) return fail(plan, PSWF_ETOLUNREACHABLE, "grid too coarse: h k_c / pi >= 1 (Nyquist criterion)");
  plan.moll = Prolate(plan.c);
  plan.est_band = std::fabs(plan.moll.eval(1.0));
  // Window bandwidth: the largest c_w whose main lobe does not alias onto the
  // band |k| < k_c: c_w = P pi (1 - eta / 2).  Spreading-error estimate
  // 10 psi_0^{c_w}(1) / eta (calibrated against the direct-sum oracle).  A
  // structure with a finer spacing than box_max gives has a smaller eta, for
  // which the same c_w and P are alias-free with more margin.
  auto cw_for = [&](int P) { return opt.c_w > 0 ? opt.c_w : P * kPi * (1.0 - 0.5 * plan.eta); };
  auto est_for = [&](const Prolate& w) { return 10.0 * std::fabs(w.eval(1.0)) / plan.eta; };
  if (opt.P > 0) {
    if (opt.P < 2 || opt.P > kMaxP) return fail(plan, PSWF_EINVAL, "P must be in 2..16");
    plan.P = opt.P;
    plan.c_w = cw_for(opt.P);
    if (!(plan.c_w > 0.0) || plan.c_w > 80.0) return fail(plan, PSWF_EINVAL, "c_w must be in (0, 80]");
    plan.win = (plan.c_w == plan.c) ? plan.moll : Prolate(plan.c_w);
  } else {
    for (int P = 2; P <= kMaxP; ++P) {
      const double cw = cw_for(P);
      if (!(cw > 0.0) || cw > 80.0) return fail(plan, PSWF_EINVAL, "c_w must be in (0, 80]");
      plan.P = P;
      plan.c_w = cw;
      plan.win = Prolate(cw);
      if (est_for(plan.win) <= opt.tol / 3.0) break;
    }
  }
  plan.est_spread = est_for(plan.win);
  for (int d = 0; d < 3; ++d) {
    plan.omega[d] = plan.P * plan.h[d] / 2.0;
    if (plan.omega[d] * plan.k_c / plan.c_w >= 1.0)
      return fail(plan, PSWF_EINVAL, "window band c_w / omega does not cover k_c");
  }
  plan.V = box_max[0] * box_max[1] * box_max[2];
  plan.dV = plan.V / (double(plan.M[0]) * plan.M[1] * plan.M[2]);
  const double eps_poly = opt.precision == 1 ? 1e-15 : 1e-9;
  // ---- window pieces: W_j(t) = psi^{c_w}((2j - P + 2t)/P), s = 2t - 1 ----
  {
    const int nfit = 41;
    std::vector<std::vector<double>> cheb(plan.P);
    const double P = plan.P;
    for (int j = 0; j < plan.P; ++j)
      cheb[j] = cheb_fit([&](double s) { return plan.win.eval((2.0 * j - P + 1.0 + s) / P); }, nfit);
    // the device pads FP32 pieces to degree 12 and FP64 pieces to 24 (FP32
    // fits need 10-12 for P >= 3; P = 2 would take 13 for 1e-9, and its
    // degree-12 fit error is still far below FP32 rounding)
    const int deg = std::min(family_degree(cheb, eps_poly), opt.precision == 1 ? kMaxDeg : 12);
    plan.deg_w = deg;
    plan.coef_w.assign(size_t(plan.P) * (deg + 1), 0.0);
    for (int j = 0; j < plan.P; ++j) {
      const auto mono = cheb_to_monomial(cheb[j], deg);
      for (int n = 0; n <= deg; ++n) plan.coef_w[size_t(j) * (deg + 1) + n] = mono[n];
    }
  }
  // ---- multiplier pieces, one row per exponent in use ----
  {
    std::vector<std::vector<double>> cheb(size_t(6) * kMultSeg);
    int deg = 1;
    for (int pp = 1; pp <= 6; ++pp) {
      if (!use_p[pp]) continue;
      const MultFit& f = mult_fit(plan.moll, pp, eps_poly);
      for (int i = 0; i < kMultSeg; ++i) cheb[size_t(pp - 1) * kMultSeg + i] = f.cheb[i];
      deg = std::max(deg, f.deg);
    }
    deg = std::min(deg, kMaxMultDeg);
    plan.deg_m = deg;
    plan.coef_m.assign(size_t(6) * kMultSeg * (deg + 1), 0.0);
    for (size_t i = 0; i < cheb.size(); ++i) {
      if (cheb[i].empty()) continue;
      const auto mono = cheb_to_monomial(cheb[i], deg);
      for (int n = 0; n <= deg; ++n) plan.coef_m[i * (deg + 1) + n] = mono[n];
    }
  }
  // ---- real-space mollifier pieces G_p(x), one row per exponent in use ----
  {
    std::vector<std::vector<double>> cheb(size_t(6) * kMultSeg);
    int deg = 1;
    for (int pp = 1; pp <= 6; ++pp) {
      if (!use_p[pp]) continue;
      const MultFit& f = real_fit(plan.moll, pp, eps_poly);
      for (int i = 0; i < kMultSeg; ++i) cheb[size_t(pp - 1) * kMultSeg + i] = f.cheb[i];
      deg = std::max(deg, f.deg);
    }
    deg = std::min(deg, kMaxMultDeg);
    plan.deg_g = deg;
    plan.coef_g.assign(size_t(6) * kMultSeg * (deg + 1), 0.0);
    for (size_t i = 0; i < cheb.size(); ++i) {
      if (cheb[i].empty()) continue;
      const auto mono = cheb_to_monomial(cheb[i], deg);
      for (int n = 0; n <= deg; ++n) plan.coef_g[i * (deg + 1) + n] = mono[n];
    }
  }
  // ---- per-exponent constants ----
  const double c = plan.c, rc = plan.r_c, C0 = plan.moll.C0, lam = plan.moll.lambda0;
  const double d2 = plan.moll.eval(0.0, 2), d4 = plan.moll.eval(0.0, 4), d6 = plan.moll.eval(0.0, 6);
  for (int pp = 1; pp <= 6; ++pp) {
    if (!use_p[pp]) continue;
    double& ms = plan.mult_scale_p[pp];
    double& sc = plan.self_coef_p[pp];
    double& zn = plan.zero_num_p[pp];
    switch (pp) {
      case 1:
        ms = 4.0 * kPi;
        sc = 1.0 / (2.0 * C0 * rc);
        // -(2 pi / V) int_0^{r_c} r (1 - G_1) dr = -(pi r_c^2 / (V C0)) int_0^1 x^2 psi
        zn = -kPi * rc * rc / C0 * plan.moll.integral(0.0, 1.0, 2);
        break;
      case 2:
        ms = 2.0 * kPi * kPi;
        sc = -d2 / (4.0 * rc * rc);
        zn = -2.0 * kPi * rc * C0;
        break;
      case 3:
        ms = 2.0 * kPi * lam / C0;
        sc = -d2 / (6.0 * C0 * rc * rc * rc);
        zn = 2.0 * kPi * (std::log(c / rc) + mult_smooth(plan.moll, 3, 0.0));
        break;
      case 4:
        ms = kPi * kPi * c / rc;
        sc = d4 / (48.0 * std::pow(rc, 4));
        zn = ms * mult_smooth(plan.moll, 4, 0.0) / 2.0;
        break;
      case 5:
        ms = -kPi * lam * c * c / (3.0 * C0 * rc * rc);
        sc = d4 / (90.0 * C0 * std::pow(rc, 5));
        zn = ms * mult_smooth(plan.moll, 5, 0.0) / 2.0;
        break;
      case 6:
        ms = kPi * kPi * c * c * c / (12.0 * rc * rc * rc);
        sc = -d6 / (1440.0 * std::pow(rc, 6));
        zn = ms * mult_smooth(plan.moll, 6, 0.0) / 2.0;
        break;
    }
  }
  return PSWF_OK;
}

}  // namespace

namespace {

// W-hat tables, scale and geometry matrices for lattice vectors H (rows).
void fill_cell_tables(const Plan& plan, const double H[9], StructTables& out) {
  const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                     H[2] * (H[3] * H[7] - H[4] * H[6]);
  // H^-1 by cofactors
  double inv[9];
  inv[0] = (H[4] * H[8] - H[5] * H[7]) / det;
  inv[1] = (H[2] * H[7] - H[1] * H[8]) / det;
  inv[2] = (H[1] * H[5] - H[2] * H[4]) / det;
  inv[3] = (H[5] * H[6] - H[3] * H[8]) / det;
  inv[4] = (H[0] * H[8] - H[2] * H[6]) / det;
  inv[5] = (H[2] * H[3] - H[0] * H[5]) / det;
  inv[6] = (H[3] * H[7] - H[4] * H[6]) / det;
  inv[7] = (H[1] * H[6] - H[0] * H[7]) / det;
  inv[8] = (H[0] * H[4] - H[1] * H[3]) / det;
  out.V = std::fabs(det);
  out.dV = 1.0;
  out.tric = false;
  for (int i = 0; i < 9; ++i) {
    out.cell[i] = H[i];
    if (i % 4 != 0 && H[i] != 0.0) out.tric = true;
  }
  for (int d = 0; d < 3; ++d) {
    const double len = std::sqrt(H[3 * d] * H[3 * d] + H[3 * d + 1] * H[3 * d + 1] + H[3 * d + 2] * H[3 * d + 2]);
    out.box[d] = len;
    out.h[d] = len / double(plan.M[d]);
    out.dV *= out.h[d];
    out.omega[d] = plan.P * out.h[d] / 2.0;
    for (int e = 0; e < 3; ++e) {
      out.tmat[3 * d + e] = double(plan.M[d]) * inv[3 * e + d];   // (H^-T)[d][e] = (H^-1)[e][d]
      out.bmat[3 * d + e] = 2.0 * kPi * inv[3 * d + e];
    }
    // the window transform per grid cell in units of h_d: k_d = 2 pi m / |a_d|
    // puts omega k_d = pi P m / M_d, independent of the cell
    const int nf = plan.M[d] / 2 + 1;
    out.iw2[d].assign(nf, 0.0);
    for (int m = 0; m < nf; ++m) {
      const double kd = 2.0 * kPi * m / len;
      const double arg = out.omega[d] * kd / plan.c_w;
      if (arg <= 1.0) {
        const double what = out.omega[d] * plan.win.lambda0 * plan.win.eval(arg);
        out.iw2[d][m] = 1.0 / (what * what);
      }
    }
  }
  if (!out.tric) {
    // an orthorhombic box: the exact products V / M and M / L, 2 pi / L
    out.V = std::fabs(H[0] * H[4] * H[8]);
    out.dV = out.V / (double(plan.M[0]) * plan.M[1] * plan.M[2]);
    for (int d = 0; d < 3; ++d) {
      out.tmat[4 * d] = double(plan.M[d]) / out.box[d];
      out.bmat[4 * d] = 2.0 * kPi / out.box[d];
    }
  }
}

}  // namespace

int struct_tables(const Plan& plan, const double box[3], StructTables& out, std::string& error) {
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0.0) || !std::isfinite(box[d])) {
      error = "box edges must be positive and finite";
      return PSWF_EINVAL;
    }
    if (box[d] > plan.box_max[d] * (1.0 + 1e-12)) {
      error = "box edge exceeds the plan's box_max";
      return PSWF_EINVAL;
    }
  }
  const double H[9] = {box[0], 0, 0, 0, box[1], 0, 0, 0, box[2]};
  fill_cell_tables(plan, H, out);
  return PSWF_OK;
}

int make_batch_plan(const double box_max[3], int K, const int* pset, int npset, const Options& opt, Plan& plan) {
  plan = Plan();
  if (npset < 1 || !pset) return fail(plan, PSWF_EINVAL, "at least one channel exponent is required");
  return plan_core(box_max, K, pset, npset, opt, plan);
}

int make_plan_cell(const double cell[9], int K, const int* p, const Options& opt, Plan& plan) {
  plan = Plan();
  if (K < 1 || K > kMaxK) return fail(plan, PSWF_EINVAL, "number of channels must be in 1..64");
  double len[3];
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) return fail(plan, PSWF_EINVAL, "cell entries must be finite");
  for (int d = 0; d < 3; ++d)
    len[d] = std::sqrt(cell[3 * d] * cell[3 * d] + cell[3 * d + 1] * cell[3 * d + 1] + cell[3 * d + 2] * cell[3 * d + 2]);
  int rc = plan_core(len, K, p, K, opt, plan);
  if (rc) return rc;
  plan.p.assign(p, p + K);
  fill_cell_tables(plan, cell, plan.st);
  if (!(plan.st.V > 1e-9 * len[0] * len[1] * len[2])) return fail(plan, PSWF_EINVAL, "cell vectors are (nearly) coplanar");
  plan.V = plan.st.V;
  for (int d = 0; d < 3; ++d) plan.iw2[d] = plan.st.iw2[d];
  plan.mult_scale.resize(K);
  plan.self_coef.resize(K);
  plan.zero_coef.resize(K);
  for (int k = 0; k < K; ++k) {
    plan.mult_scale[k] = plan.mult_scale_p[p[k]];
    plan.self_coef[k] = plan.self_coef_p[p[k]];
    plan.zero_coef[k] = plan.zero_num_p[p[k]] / plan.V;
  }
  return PSWF_OK;
}

int make_plan(const double box[3], int K, const int* p, const Options& opt, Plan& plan) {
  plan = Plan();
  if (K < 1 || K > kMaxK) return fail(plan, PSWF_EINVAL, "number of channels must be in 1..64");
  int rc = plan_core(box, K, p, K, opt, plan);
  if (rc) return rc;
  plan.p.assign(p, p + K);
  if ((rc = struct_tables(plan, box, plan.st, plan.error))) return rc;
  for (int d = 0; d < 3; ++d) plan.iw2[d] = plan.st.iw2[d];
  plan.mult_scale.resize(K);
  plan.self_coef.resize(K);
  plan.zero_coef.resize(K);
  for (int k = 0; k < K; ++k) {
    plan.mult_scale[k] = plan.mult_scale_p[p[k]];
    plan.self_coef[k] = plan.self_coef_p[p[k]];
    plan.zero_coef[k] = plan.zero_num_p[p[k]] / plan.V;
  }
  return PSWF_OK;
}

}  // namespace pswf
