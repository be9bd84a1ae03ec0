// Host planner for PSWF-LR (FP64, no CUDA).
//
// Computes, once per plan, every constant the device kernels need:
//   * psi_0^c and psi_0^{c_w} (Methods, "Prolate spheroidal wave functions"),
//     here by the Legendre expansion of the prolate differential operator
//     that commutes with F_c;
//   * the parameters of "Parameter selection" (c, k_c, h, M_d, P) and the
//     window bandwidth c_w;
//   * the Horner piecewise polynomials of the spreading window W_pswf and of
//     the smooth parts of Phi-hat_p (Methods, "Implementation details": FKAD,
//     Chebyshev-coefficient filtering then monomial conversion);
//   * the 1-D tables of W-hat_pswf(k_d)^-2 (Eq. EthetaLR);
//   * self-energy and zero-frequency coefficients ("Implementation details").
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace pswf {

constexpr int kMaxP = 16;        // largest stencil width
constexpr int kMaxDeg = 24;      // largest window polynomial degree
constexpr int kMultSeg = 32;     // pieces of the multiplier polynomial on [0,1]
constexpr int kMaxMultDeg = 16;  // largest multiplier polynomial degree
constexpr int kMaxK = 64;        // largest number of channels

// psi_0^c as a Legendre series psi(x) = sum_k beta_k Pbar_{2k}(x), scaled so
// that psi(0) = 1 (Pbar_n = sqrt(n + 1/2) P_n).
struct Prolate {
  double c = 0.0;
  double chi = 0.0;       // eigenvalue of the prolate differential operator
  double lambda0 = 0.0;   // eigenvalue of F_c, = int_{-1}^{1} psi
  double C0 = 0.0;        // int_0^1 psi
  std::vector<double> beta;
  std::vector<double> bs;  // beta_k sqrt(2k + 1/2): psi = sum_k bs_k P_{2k}

  explicit Prolate(double c_);
  Prolate() = default;
  // m-th derivative of psi at x (m <= 8), any real x.
  double eval(double x, int m = 0) const;
  // int_a^b s^power psi(s) ds (Gauss-Legendre, 64 nodes).
  double integral(double a, double b, int power = 0) const;
};

// Gauss-Legendre rule on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// Smallest integer >= n whose prime factors are all in {2, 3, 5, 7}.
int64_t next_fft_size(int64_t n);

struct Options {
  double tol = 1e-5;      // target LR tolerance epsilon_tot
  double r_c = 0.0;       // mollifier cutoff (required)
  double c = 0.0;         // 0 -> log(3 / tol)
  double c_w = 0.0;       // 0 -> P pi (1 - eta / 2)
  double eta = 0.0;       // 0 -> 0.5
  int P = 0;              // 0 -> smallest P meeting tol / 3
  int grid[3] = {0, 0, 0};
  int precision = 0;      // 0 fp32 path, 1 fp64 path
};

// Cell-dependent tables of one structure on a plan's grid.  The cell's
// lattice vectors a_d are the rows of H (an orthorhombic box: H = diag(L));
// the grid is uniform in the fractional coordinates, u_d = M_d s_d.
struct StructTables {
  double box[3] = {0, 0, 0};       // edge lengths |a_d|
  double h[3] = {0, 0, 0};         // |a_d| / M_d
  double omega[3] = {0, 0, 0};     // P h_d / 2
  double V = 0;                    // |det H|
  double dV = 0;                   // prod_d h_d (= V / M for a box): the multiplier scale is dV^2 / V
  std::vector<double> iw2[3];      // (h_d W-hat_d)^-2 by |frequency| (0 .. M_d/2)
  double cell[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // H, row-major
  double tmat[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // T = diag(M) H^-T: u = T r
  double bmat[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // B = 2 pi H^-1: k_m = B m
  bool tric = false;                              // H has off-diagonal entries
};

struct Plan {
  // inputs
  double box[3] = {0, 0, 0};       // the box of a single-structure plan
  double box_max[3] = {0, 0, 0};   // largest box a structure of this plan may have
  int K = 0;
  std::vector<int> p;              // exponent per channel (single-structure plans)
  Options opt;
  // chosen parameters (h, omega, eta: at box_max)
  double c = 0, c_w = 0, r_c = 0, k_c = 0, eta = 0, tol = 0;
  double h[3] = {0, 0, 0};
  double omega[3] = {0, 0, 0};
  int M[3] = {0, 0, 0};
  int P = 0;
  double V = 0, dV = 0;
  double est_spread = 0, est_band = 0;
  Prolate moll;                  // psi_0^c
  Prolate win;                   // psi_0^{c_w}
  // window pieces: coef_w[j][n], monomials in s = 2t - 1, j = 0..P-1
  int deg_w = 0;
  std::vector<double> coef_w;    // P * (deg_w + 1)
  // multiplier smooth parts: per exponent p (row p - 1; rows of exponents the
  // plan does not use are zero), kMultSeg pieces on u in [0, 1]
  int deg_m = 0;
  std::vector<double> coef_m;    // 6 * kMultSeg * (deg_m + 1)
  // real-space mollifier G_p(x), x = r / r_c: same piece layout in x as the
  // multiplier (row p - 1), for the real-space complement (1 - G_p) / r^p
  int deg_g = 0;
  std::vector<double> coef_g;    // 6 * kMultSeg * (deg_g + 1)
  // per exponent p (index p, 1..6): constant in front of S_p, self-energy
  // coefficient, and V times the zero-frequency coefficient
  double mult_scale_p[7] = {0, 0, 0, 0, 0, 0, 0};
  double self_coef_p[7] = {0, 0, 0, 0, 0, 0, 0};
  double zero_num_p[7] = {0, 0, 0, 0, 0, 0, 0};
  // tables of the single-structure box (box == box_max)
  StructTables st;
  std::vector<double> iw2[3];      // = st.iw2
  std::vector<double> mult_scale;  // per channel
  std::vector<double> self_coef;   // E_self = self_coef * sum q^2, per channel
  std::vector<double> zero_coef;   // E^0 = zero_coef * Q_net^2, per channel
  std::string error;
};

// Returns 0 on success, or a negative pswf status with plan.error set.
// Single structure: the grid, stencil and window are chosen for `box`.
int make_plan(const double box[3], int K, const int* p, const Options& opt, Plan& plan);

// Batch of structures sharing one grid: parameters chosen at `box_max` (the
// coarsest spacing any structure will have), multiplier tables built for the
// exponents in pset[0 .. npset-1]; plan.p stays empty.
int make_batch_plan(const double box_max[3], int K, const int* pset, int npset, const Options& opt, Plan& plan);

// Tables of one structure with edges `box` (each <= box_max) on the plan's grid.
int struct_tables(const Plan& plan, const double box[3], StructTables& out, std::string& error);

// Single structure in a general (triclinic) cell: lattice vectors as the rows
// of cell[9] (right-handed or not; V = |det|).  Grid, stencil and window are
// chosen for the edge lengths |a_d| (the spacing that bounds the band's
// extent in each grid direction is |a_d| / M_d).
int make_plan_cell(const double cell[9], int K, const int* p, const Options& opt, Plan& plan);

// Smooth part S_p(u) of Phi-hat_p = mult_scale_p * singular_p(k) * S_p(u),
// u = k / k_c in [0, 1] (host FP64 reference used to fit the polynomials).
double mult_smooth(const Prolate& ps, int p, double u);

}  // namespace pswf
