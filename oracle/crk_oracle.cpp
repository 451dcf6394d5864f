// crk_oracle.cpp -- plain FP64 CPU oracle for the CRKSPH neighbor-sum path.
//
// TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU
// baseline leg call this file; the product path (the CUDA library) never does,
// and the two share no code, header, table or helper.
//
// What it computes (CRK-HACC, arXiv 2511.21921, and the CRKSPH formulation that
// paper cites for the parts it does not print):
//   * Wendland C4 kernel with compact support h (Sec. 2 preamble; App. A.2 footnote on
//     the radius convention).
//   * gas volume  V_i = m_i / sum_j m_j W(|x_ij|, h_i)            (App. A.2, Eq. Vg)
//   * geometric moments m0, m1, m2 and their gradients, and the reproducing
//     kernel coefficients A, B, grad A, grad B, obtained by imposing that the
//     corrected kernel reproduces constant and linear fields   (App. A.1, Eq. RK;
//     the paper defers the closed forms to the CRKSPH method paper)
//   * corrected kernel W^R_ij = A_i (1 + B_i . x_ij) W_ij(h_i)    (App. A.1, Eq. RK)
//   * gas density  rho_i = sum m_j V_j W^R_ij / sum V_j^2 W^R_ij  (Sec. 2.5.1, Eq. rhow,
//     gas-only)
//   * velocity gradient  grad v_i = -sum_j V_j (v_i - v_j) (x) grad W^R_ij (App. A.1, Eq. gradv)
//   * ideal-gas EOS with gamma = 5/3                              (Sec. 2.4.1)
//   * RK relaxation: exp(|div v_i| dt) > 8 => A=1, B=0 for any pair with that
//     particle, applied symmetrically                            (App. A.1)
//   * pairwise momentum and compatible-energy rates with a limited
//     artificial viscosity                                       (Sec. 2.1; App. A.1 limiter)
//
// Precision: double throughout, compiled with -ffp-contract=off (no FMA), so
// every product and sum is rounded exactly as written.  The scalar type is a
// template parameter; instantiating it with a forward-mode dual number gives a
// Jacobian-vector product of the whole chain with no separate derivative code.
//
// Pins (tests/): kernel quadrature and derivative, brute-force neighbor sets,
// reproduction identities, lattice symmetries, exact gradients of linear
// fields, conservation with equal and unequal masses, the mass linearity of
// the volume and the closed-form density on a two-species lattice, the
// standard-SPH reduction, and the linear-field limiter tests (phi(1) = 1, the
// limited relative velocity vanishes, damping only below eta_crit).
// Parity unpinned: the shape of the limiter phi(r) away from r = 1 and the
// viscosity constants are readings of the cited formulation, fixed by no
// printed value; the GPU path must match this file there.
//
// Plainness: every stage is the definition written out as a loop over the
// neighbor set of one particle.  Neighbor sets come from brute force (O(N^2))
// or from a simple k-d tree whose leaves apply the same exact predicate; the
// tests check that the two agree bit for bit.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <numeric>
#include <array>
#include <functional>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ----------------------------------------------------------------------------
// forward-mode dual number (value, one tangent)
// ----------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  // sqrt is only ever applied to r^2 (zero only for the self pair, whose
  // tangent is identically zero) and to gamma(gamma-1)u (> 0).
  return {s, s > 0 ? a.d / (2 * s) : 0.0};
}
inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, e * a.d}; }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
inline double tan_of(double) { return 0.0; }
inline double tan_of(const Dual& a) { return a.d; }

// ----------------------------------------------------------------------------
// operation counting (the algorithmic flop counts of the benchmark): a value
// type that counts every add, subtract, multiply, divide, square root and
// exponential it performs (one each), and a dual number that counts the
// operations on its value and on its tangent separately.  Comparisons and
// selections count nothing.  The counters are per thread; counting runs on
// one thread.
// ----------------------------------------------------------------------------
thread_local int64_t g_val_ops = 0, g_tan_ops = 0;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double a) : v(a) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_val_ops; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_val_ops; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_val_ops; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_val_ops; return Cnt(a.v / b.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline Cnt sqrt(Cnt a) { ++g_val_ops; return Cnt(std::sqrt(a.v)); }
inline Cnt exp(Cnt a) { ++g_val_ops; return Cnt(std::exp(a.v)); }
inline double val(const Cnt& a) { return a.v; }
inline double tan_of(const Cnt&) { return 0.0; }

// a dual number counting value operations (as Cnt) and tangent operations:
// d(a+b) 1, d(ab) 3, d(a/b) 3 (reusing the quotient), d sqrt 2, d exp 1
struct CDual {
  Dual x;
  CDual() {}
  CDual(double a) : x(a) {}
  CDual(double a, double b) : x(a, b) {}
  CDual(Dual d) : x(d) {}
};
inline CDual operator+(CDual a, CDual b) { ++g_val_ops; ++g_tan_ops; return CDual(a.x + b.x); }
inline CDual operator-(CDual a, CDual b) { ++g_val_ops; ++g_tan_ops; return CDual(a.x - b.x); }
inline CDual operator-(CDual a) { return CDual(-a.x); }
inline CDual operator*(CDual a, CDual b) { ++g_val_ops; g_tan_ops += 3; return CDual(a.x * b.x); }
inline CDual operator/(CDual a, CDual b) { ++g_val_ops; g_tan_ops += 3; return CDual(a.x / b.x); }
inline CDual& operator+=(CDual& a, CDual b) { a = a + b; return a; }
inline CDual& operator-=(CDual& a, CDual b) { a = a - b; return a; }
inline CDual& operator*=(CDual& a, CDual b) { a = a * b; return a; }
inline CDual sqrt(CDual a) { ++g_val_ops; g_tan_ops += 2; return CDual(sqrt(a.x)); }
inline CDual exp(CDual a) { ++g_val_ops; g_tan_ops += 1; return CDual(exp(a.x)); }
inline double val(const CDual& a) { return a.x.v; }
inline double tan_of(const CDual& a) { return a.x.d; }

template <class T> inline T tmax(T a, T b) { return val(a) >= val(b) ? a : b; }
template <class T> inline T tmin(T a, T b) { return val(a) <= val(b) ? a : b; }
template <class T> inline T tabs(T a) { return val(a) < 0 ? T(0) - a : a; }
using std::sqrt;
using std::exp;

// ----------------------------------------------------------------------------
// periodic minimum image and the exact pair predicate (double only)
// ----------------------------------------------------------------------------
// dx = x_i - x_j; if dx > L/2: dx -= L; elif dx < -L/2: dx += L (a tie at
// exactly +-L/2 is left unchanged).  Returns the shift that was added.
inline double image_shift(double d, double L) {
  const double half = 0.5 * L;
  if (d > half) return -L;
  if (d < -half) return L;
  return 0.0;
}
inline double min_image(double d, double L) { return d + image_shift(d, L); }

struct Box {
  int64_t n;
  const double* x;  // [3][n]
  const double* h;  // [n]
  double L;
  double r2(int64_t i, int64_t j) const {
    double dx = min_image(x[i] - x[j], L);
    double dy = min_image(x[n + i] - x[n + j], L);
    double dz = min_image(x[2 * n + i] - x[2 * n + j], L);
    return dx * dx + dy * dy + dz * dz;
  }
  // gather set G(i): r^2 < h_i^2, self included
  bool in_gather(int64_t i, int64_t j) const { return r2(i, j) < h[i] * h[i]; }
  // union set U(i): j != i and r^2 < max(h_i, h_j)^2
  bool in_union(int64_t i, int64_t j) const {
    if (i == j) return false;
    double q = r2(i, j);
    return q < h[i] * h[i] || q < h[j] * h[j];
  }
};

// ----------------------------------------------------------------------------
// neighbor search: brute force and a plain k-d tree (same leaf predicate)
// ----------------------------------------------------------------------------
struct KDTree {
  const Box* b;
  std::vector<int64_t> idx;
  struct Node {
    double lo[3], hi[3], hmax;
    int64_t begin, end;
    int64_t left, right;
  };
  std::vector<Node> nodes;

  explicit KDTree(const Box* box) : b(box) {
    idx.resize(b->n);
    std::iota(idx.begin(), idx.end(), 0);
    if (b->n > 0) build(0, b->n);
  }
  int64_t build(int64_t begin, int64_t end) {
    Node nd;
    for (int a = 0; a < 3; ++a) { nd.lo[a] = INFINITY; nd.hi[a] = -INFINITY; }
    nd.hmax = 0;
    for (int64_t k = begin; k < end; ++k) {
      int64_t p = idx[k];
      for (int a = 0; a < 3; ++a) {
        nd.lo[a] = std::min(nd.lo[a], b->x[a * b->n + p]);
        nd.hi[a] = std::max(nd.hi[a], b->x[a * b->n + p]);
      }
      nd.hmax = std::max(nd.hmax, b->h[p]);
    }
    nd.begin = begin; nd.end = end; nd.left = nd.right = -1;
    int64_t me = (int64_t)nodes.size();
    nodes.push_back(nd);
    if (end - begin > 8) {
      int ax = 0;
      for (int a = 1; a < 3; ++a)
        if (nd.hi[a] - nd.lo[a] > nd.hi[ax] - nd.lo[ax]) ax = a;
      int64_t mid = (begin + end) / 2;
      const double* xa = b->x + ax * b->n;
      std::nth_element(idx.begin() + begin, idx.begin() + mid, idx.begin() + end,
                       [xa](int64_t p, int64_t q) { return xa[p] < xa[q]; });
      int64_t l = build(begin, mid);
      int64_t r = build(mid, end);
      nodes[me].left = l; nodes[me].right = r;
    }
    return me;
  }
  // Periodic distance from point i to the node's box, per axis: the gap
  // between the point and the interval [lo, hi] under the minimum image.
  double gap2(int64_t i, const Node& nd) const {
    double g2 = 0;
    for (int a = 0; a < 3; ++a) {
      double c = 0.5 * (nd.lo[a] + nd.hi[a]);
      double e = 0.5 * (nd.hi[a] - nd.lo[a]);
      double d = std::fabs(min_image(b->x[a * b->n + i] - c, b->L)) - e;
      if (d > 0) g2 += d * d;
    }
    return g2;
  }
  // Collect every j with pred(i, j); prune a node only when no point in it can
  // be within the search radius (conservative margin against rounding).
  template <class Pred>
  void query(int64_t i, bool use_union, Pred pred, std::vector<int64_t>& out) const {
    if (nodes.empty()) return;
    std::vector<int64_t> stack;
    stack.push_back(0);
    const double hi_ = b->h[i];
    while (!stack.empty()) {
      const Node& nd = nodes[stack.back()];
      stack.pop_back();
      double R = use_union ? std::max(hi_, nd.hmax) : hi_;
      if (gap2(i, nd) > R * R * (1.0 + 1e-9)) continue;
      if (nd.left < 0) {
        for (int64_t k = nd.begin; k < nd.end; ++k)
          if (pred(i, idx[k])) out.push_back(idx[k]);
      } else {
        stack.push_back(nd.left);
        stack.push_back(nd.right);
      }
    }
    std::sort(out.begin(), out.end());
  }
};

// ----------------------------------------------------------------------------
// Wendland C4 kernel in 3-D with compact support h (q = r/h < 1):
//   W(r, h)      = 495/(32 pi h^3) (1-q)^6 (1 + 6q + 35 q^2 / 3)
//   dW/dr        = 495/(32 pi h^4) (-56/3) q (1-q)^5 (1 + 5q)
//   g(r, h) = (1/r) dW/dr = 495/(32 pi h^5) (-56/3) (1-q)^5 (1 + 5q)
// so that grad W = g(r, h) x_ij, smooth at r = 0.
// ----------------------------------------------------------------------------
const double kWendC4 = 495.0 / (32.0 * M_PI);

template <class T> T kernel_W(T r, T h) {
  T q = r / h;
  if (val(q) >= 1.0) return T(0.0);
  T om = T(1.0) - q;
  T om2 = om * om;
  T om6 = om2 * om2 * om2;
  return T(kWendC4) / (h * h * h) * om6 * (T(1.0) + T(6.0) * q + T(35.0 / 3.0) * q * q);
}
template <class T> T kernel_dWdr(T r, T h) {
  T q = r / h;
  if (val(q) >= 1.0) return T(0.0);
  T om = T(1.0) - q;
  T om2 = om * om;
  T om5 = om2 * om2 * om;
  return T(kWendC4) / (h * h * h * h) * T(-56.0 / 3.0) * q * om5 * (T(1.0) + T(5.0) * q);
}
template <class T> T kernel_g(T r, T h) {
  T q = r / h;
  if (val(q) >= 1.0) return T(0.0);
  T om = T(1.0) - q;
  T om2 = om * om;
  T om5 = om2 * om2 * om;
  T h2 = h * h;
  return T(kWendC4) / (h2 * h2 * h) * T(-56.0 / 3.0) * om5 * (T(1.0) + T(5.0) * q);
}

}  // namespace

extern "C" {

typedef struct {
  double gamma;     // adiabatic index (5/3, Sec. 2.4.1)
  double Cl, Cq;    // linear and quadratic viscosity coefficients
  double eps2;      // softening of the viscosity denominator
  double eta_crit;  // near-field damping threshold on r/h
  double eta_fold;  // near-field damping width
  double relax_dt;  // relaxation time step; 0 turns relaxation off (App. A.1)
  int32_t limiter;  // 1: limited viscosity, 0: unlimited
  int32_t energy_split;  // 0: f_ij = 1/2; 1: weighted by the specific energies
  int32_t q_side;   // 0: Q_ij + Q_ji with the pressures; 1: each Q with its own gradient
  int32_t pad;
} oracle_params;

typedef struct {
  double* V;        // [nt]
  double* coef;     // [16][nt]: A, B[3], gradA[3], gradB[3][3] ([gamma][alpha])
  double* mom;      // [40][nt]: m0, m1[3], m2[6], dm0[3], dm1[3][3], dm2[3][6]
  double* rho;      // [nt]
  double* gradv;    // [9][nt]: (grad v)^{ab} = d v^a / d x^b, index a*3+b
  double* P;        // [nt]
  double* cs;       // [nt]
  int8_t* flag;     // [nt] relaxation flag
  double* dvdt;     // [3][nt]
  double* dudt;     // [nt]
  int64_t* kgather; // [nt] |G(i)| - 1 (neighbors excluding self)
  int64_t* kunion;  // [nt] |U(i)|
  double* diag;     // [16][nt] reproduction diagnostics: sum V W^R, sum V W^R x[3],
                    //   sum V gradW^R[3], sum V x (x) gradW^R [3][3]
  int64_t* nsingular;  // scalar: particles whose m2 was singular
} oracle_out;

}  // extern "C"

namespace {

enum { OK = 0, EINVAL_ = 1, EDOMAIN_ = 4, ENONFINITE_ = 5, ESINGULAR_ = 6 };

// symmetric 3x3 index for (a, b) into the 6-vector xx, xy, xz, yy, yz, zz
inline int sym6(int a, int b) {
  static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return t[a][b];
}

template <class T>
struct Eval {
  const Box& box;
  const KDTree* tree;
  const oracle_params& p;
  int64_t n;
  double L;
  // inputs (scalar type T carries tangents for the JVP)
  std::vector<T> x[3], h, m, v[3], u;
  // neighbor lists (memoised)
  std::vector<std::vector<int64_t>> G, U;
  std::vector<char> hasG, hasU;
  // species: 0 gas, 1 wind (Sec. 2.5.1: winds enter the gas density, Eq. rhow,
  // but no hydrodynamic force); empty = all gas
  std::vector<uint8_t> sp;
  bool wind(int64_t j) const { return !sp.empty() && sp[j] != 0; }
  // per-particle stage results (memoised)
  std::vector<T> V, Vgw;
  std::vector<std::array<T, 40>> mom;
  std::vector<std::array<T, 16>> coef;
  std::vector<T> rho, P, cs;
  std::vector<std::array<T, 9>> gradv;
  std::vector<char> flag;
  std::vector<char> doneV, doneM, doneR, sing;

  Eval(const Box& b, const KDTree* t, const oracle_params& pp)
      : box(b), tree(t), p(pp), n(b.n), L(b.L) {
    for (int a = 0; a < 3; ++a) { x[a].resize(n); v[a].resize(n); }
    h.resize(n); m.resize(n); u.resize(n);
    G.resize(n); U.resize(n); hasG.assign(n, 0); hasU.assign(n, 0);
    V.resize(n); Vgw.resize(n); mom.resize(n); coef.resize(n);
    rho.resize(n); P.resize(n); cs.resize(n); gradv.resize(n); flag.assign(n, 0);
    doneV.assign(n, 0); doneM.assign(n, 0); doneR.assign(n, 0); sing.assign(n, 0);
  }

  const std::vector<int64_t>& gather(int64_t i) {
    if (!hasG[i]) {
      std::vector<int64_t> out;
      auto pred = [this](int64_t a, int64_t c) { return box.in_gather(a, c); };
      if (tree) tree->query(i, false, pred, out);
      else for (int64_t j = 0; j < n; ++j) if (pred(i, j)) out.push_back(j);
      G[i].swap(out);
      hasG[i] = 1;
    }
    return G[i];
  }
  const std::vector<int64_t>& unionset(int64_t i) {
    if (!hasU[i]) {
      std::vector<int64_t> out;
      auto pred = [this](int64_t a, int64_t c) { return box.in_union(a, c); };
      if (tree) tree->query(i, true, pred, out);
      else for (int64_t j = 0; j < n; ++j) if (pred(i, j)) out.push_back(j);
      U[i].swap(out);
      hasU[i] = 1;
    }
    return U[i];
  }

  // x_ij = x_i - x_j under the minimum image.  The image shift is decided on the
  // double values and held fixed, so a tangent passes through it unchanged.
  void sep(int64_t i, int64_t j, T out[3]) const {
    for (int a = 0; a < 3; ++a) {
      double s = image_shift(box.x[a * n + i] - box.x[a * n + j], L);
      out[a] = (x[a][i] - x[a][j]) + T(s);
    }
  }
  static T dot3(const T a[3], const T b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

  // ---- volume, Eq. Vg:  V_i = m_i / sum_{j in G(i), gas} m_j W(r_ij, h_i), and
  // the volume over gas and wind neighbors, V_{g+w} (App. A.2), that the
  // density uses.  A wind particle's V is its V_{g+w} (it takes no part in the
  // gas-only sums).
  void calcV(int64_t i) {
    const auto& nb = gather(i);
    T s(0.0), sa(0.0);
    for (int64_t j : nb) {
      T xij[3];
      sep(i, j, xij);
      T r = (j == i) ? T(0.0) : sqrt(dot3(xij, xij));
      T w = m[j] * kernel_W(r, h[i]);
      if (!wind(j)) s += w;
      sa += w;
    }
    Vgw[i] = m[i] / sa;
    V[i] = wind(i) ? Vgw[i] : m[i] / s;
    doneV[i] = 1;
  }
  void ensureV(int64_t i) { if (!doneV[i]) calcV(i); }

  // ---- moments and their gradients (V_j held constant), over G(i):
  //   m0 = sum V_j W, m1^a = sum V_j x^a W, m2^ab = sum V_j x^a x^b W
  //   d_g m0 = sum V_j d_gW
  //   d_g m1^a = sum V_j (x^a d_gW + delta_ag W)
  //   d_g m2^ab = sum V_j (x^a x^b d_gW + (delta_ag x^b + delta_bg x^a) W)
  // where d_gW = g(r, h_i) x^g is the gradient with respect to x_i.
  void calcMom(int64_t i) {
    const auto& nb = gather(i);
    std::array<T, 40> M;
    for (auto& e : M) e = T(0.0);
    T* m0 = &M[0]; T* m1 = &M[1]; T* m2 = &M[4];
    T* dm0 = &M[10]; T* dm1 = &M[13]; T* dm2 = &M[22];
    for (int64_t j : nb) {
      if (wind(j)) continue;  // the corrections reproduce over the gas
      ensureV(j);
      T xij[3];
      sep(i, j, xij);
      T r = (j == i) ? T(0.0) : sqrt(dot3(xij, xij));
      T W = kernel_W(r, h[i]);
      T gr = kernel_g(r, h[i]);
      T dW[3] = {gr * xij[0], gr * xij[1], gr * xij[2]};
      const T& Vj = V[j];
      m0[0] += Vj * W;
      for (int a = 0; a < 3; ++a) m1[a] += Vj * xij[a] * W;
      for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) m2[sym6(a, b)] += Vj * xij[a] * xij[b] * W;
      for (int g = 0; g < 3; ++g) dm0[g] += Vj * dW[g];
      for (int g = 0; g < 3; ++g)
        for (int a = 0; a < 3; ++a) {
          T t = xij[a] * dW[g];
          if (a == g) t += W;
          dm1[g * 3 + a] += Vj * t;
        }
      for (int g = 0; g < 3; ++g)
        for (int a = 0; a < 3; ++a)
          for (int b = a; b < 3; ++b) {
            T t = xij[a] * xij[b] * dW[g];
            if (a == g) t += xij[b] * W;
            if (b == g) t += xij[a] * W;
            dm2[g * 6 + sym6(a, b)] += Vj * t;
          }
    }
    mom[i] = M;
    calcCoef(i);
    doneM[i] = 1;
  }
  void ensureMom(int64_t i) { if (!doneM[i]) calcMom(i); }

  // ---- coefficients from the reproducing conditions
  //   sum V_j W^R_ij = 1,  sum V_j W^R_ij x_ij = 0,  W^R = A (1 + B.x) W:
  //   M = m2^{-1}; B = -M m1; A = 1 / (m0 - m1.M m1)
  //   d_g A = -A^2 (d_g m0 - 2 m1.M d_g m1 + m1.M (d_g m2) M m1)
  //   d_g B = -M d_g m1 + M (d_g m2) M m1
  void calcCoef(int64_t i) {
    const auto& Mo = mom[i];
    const T& m0 = Mo[0];
    T m1[3] = {Mo[1], Mo[2], Mo[3]};
    T m2[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) m2[a][b] = Mo[4 + sym6(a, b)];
    // inverse by cofactors
    T c00 = m2[1][1] * m2[2][2] - m2[1][2] * m2[2][1];
    T c01 = m2[1][2] * m2[2][0] - m2[1][0] * m2[2][2];
    T c02 = m2[1][0] * m2[2][1] - m2[1][1] * m2[2][0];
    T det = m2[0][0] * c00 + m2[0][1] * c01 + m2[0][2] * c02;
    double tr = std::fabs(val(m2[0][0])) + std::fabs(val(m2[1][1])) + std::fabs(val(m2[2][2]));
    std::array<T, 16> C;
    if (!(std::fabs(val(det)) > 1e-12 * (tr / 3) * (tr / 3) * (tr / 3))) {
      // singular second moment: fall back to the uncorrected kernel
      C[0] = T(1.0);
      for (int k = 1; k < 16; ++k) C[k] = T(0.0);
      coef[i] = C;
      sing[i] = 1;
      return;
    }
    T Mi[3][3];
    Mi[0][0] = c00 / det; Mi[1][0] = c01 / det; Mi[2][0] = c02 / det;
    Mi[0][1] = (m2[0][2] * m2[2][1] - m2[0][1] * m2[2][2]) / det;
    Mi[1][1] = (m2[0][0] * m2[2][2] - m2[0][2] * m2[2][0]) / det;
    Mi[2][1] = (m2[0][1] * m2[2][0] - m2[0][0] * m2[2][1]) / det;
    Mi[0][2] = (m2[0][1] * m2[1][2] - m2[0][2] * m2[1][1]) / det;
    Mi[1][2] = (m2[0][2] * m2[1][0] - m2[0][0] * m2[1][2]) / det;
    Mi[2][2] = (m2[0][0] * m2[1][1] - m2[0][1] * m2[1][0]) / det;
    T Mm1[3];
    for (int a = 0; a < 3; ++a) Mm1[a] = Mi[a][0] * m1[0] + Mi[a][1] * m1[1] + Mi[a][2] * m1[2];
    T B[3] = {T(0.0) - Mm1[0], T(0.0) - Mm1[1], T(0.0) - Mm1[2]};
    T A = T(1.0) / (m0 - dot3(m1, Mm1));
    T dA[3], dB[3][3];
    for (int g = 0; g < 3; ++g) {
      T d1[3] = {Mo[13 + g * 3 + 0], Mo[13 + g * 3 + 1], Mo[13 + g * 3 + 2]};
      T d2[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) d2[a][b] = Mo[22 + g * 6 + sym6(a, b)];
      // t = d_g m2 (M m1)
      T t[3];
      for (int a = 0; a < 3; ++a) t[a] = d2[a][0] * Mm1[0] + d2[a][1] * Mm1[1] + d2[a][2] * Mm1[2];
      // d_g A
      T s = Mo[10 + g] - T(2.0) * dot3(Mm1, d1) + dot3(Mm1, t);
      dA[g] = T(0.0) - A * A * s;
      // d_g B = M (t - d1)
      T w[3] = {t[0] - d1[0], t[1] - d1[1], t[2] - d1[2]};
      for (int a = 0; a < 3; ++a) dB[g][a] = Mi[a][0] * w[0] + Mi[a][1] * w[1] + Mi[a][2] * w[2];
    }
    C[0] = A;
    for (int a = 0; a < 3; ++a) C[1 + a] = B[a];
    for (int g = 0; g < 3; ++g) C[4 + g] = dA[g];
    for (int g = 0; g < 3; ++g)
      for (int a = 0; a < 3; ++a) C[7 + g * 3 + a] = dB[g][a];
    coef[i] = C;
  }

  // ---- corrected kernel and its gradient for particle k (its h_k and
  // coefficients) at separation xx = x_k - x_j:
  //   W^R = A (1 + B.x) W
  //   grad W^R = gradA (1 + B.x) W + A (gradB.x + B) W + A (1 + B.x) grad W
  // with (gradB.x)_g = sum_a d_g B^a x^a.  With corrected == false the pair
  // uses A = 1, B = 0 (relaxation).
  void corrected(int64_t k, const T xx[3], bool self, bool corrected_kernel, T& WR, T Gr[3]) {
    T r = self ? T(0.0) : sqrt(dot3(xx, xx));
    T W = kernel_W(r, h[k]);
    T gr = kernel_g(r, h[k]);
    T dW[3] = {gr * xx[0], gr * xx[1], gr * xx[2]};
    if (!corrected_kernel) {
      WR = W;
      for (int g = 0; g < 3; ++g) Gr[g] = dW[g];
      return;
    }
    const auto& C = coef[k];
    const T& A = C[0];
    T B[3] = {C[1], C[2], C[3]};
    T lin = T(1.0) + dot3(B, xx);
    WR = A * lin * W;
    for (int g = 0; g < 3; ++g) {
      T dBx = C[7 + g * 3 + 0] * xx[0] + C[7 + g * 3 + 1] * xx[1] + C[7 + g * 3 + 2] * xx[2];
      Gr[g] = C[4 + g] * lin * W + A * (dBx + B[g]) * W + A * lin * dW[g];
    }
  }

  // ---- density (Eq. rhow, gas only) and velocity gradient (Eq. gradv), EOS,
  // relaxation flag
  void calcRho(int64_t i) {
    ensureMom(i);
    const auto& nb = gather(i);
    T num(0.0), den(0.0);
    std::array<T, 9> gv;
    for (auto& e : gv) e = T(0.0);
    for (int64_t j : nb) {
      ensureV(j);
      T xij[3];
      sep(i, j, xij);
      T WR, Gr[3];
      corrected(i, xij, j == i, true, WR, Gr);
      // density over gas and wind (Eq. rhow) with V_{g+w}; velocity gradient
      // over the gas (Eq. gradv)
      num += m[j] * Vgw[j] * WR;
      den += Vgw[j] * Vgw[j] * WR;
      if (wind(j)) continue;
      for (int a = 0; a < 3; ++a) {
        T dv = v[a][i] - v[a][j];
        for (int b = 0; b < 3; ++b) gv[a * 3 + b] -= V[j] * dv * Gr[b];
      }
    }
    rho[i] = num / den;
    gradv[i] = gv;
    P[i] = T(p.gamma - 1.0) * rho[i] * u[i];
    cs[i] = sqrt(T(p.gamma * (p.gamma - 1.0)) * u[i]);
    double div = val(gv[0]) + val(gv[4]) + val(gv[8]);
    flag[i] = (p.relax_dt > 0 && std::exp(std::fabs(div) * p.relax_dt) > 8.0) ? 1 : 0;
    doneR[i] = 1;
  }
  void ensureRho(int64_t i) { if (!doneR[i]) calcRho(i); }

  // ---- pair rates over the union set U(i), each ordered pair from i's side:
  //   G_ij = grad W^R_ij (i's coefficients, h_i); G_ji likewise with j's and x_ji
  //   limited viscosity Q_ij, Q_ji; Pi = P_i + P_j + Q_ij + Q_ji
  //   m_i a_ij = -(1/2) V_i V_j Pi (G_ij - G_ji)
  //   or, with q_side, each side's viscosity with its own gradient:
  //   m_i a_ij = -(1/2) V_i V_j [(P_i + P_j)(G_ij - G_ji) + 2 (Q_ij G_ij - Q_ji G_ji)]
  //   (both antisymmetric in i, j; equal when Q_ij = Q_ji)
  //   pair work E_ij = m_i a_ij . (v_j - v_i) (symmetric in i, j)
  //   dv_i/dt = sum_j a_ij;  du_i/dt = (1/m_i) sum_j f_ij E_ij
  //   compatible split (Sec. 2.1): f_ij + f_ji = 1, so the pair's thermal energy
  //   change is its kinetic energy loss.  f_ij = 1/2, or with energy_split
  //   f_ij = (1/2)(1 + sgn(E_ij) (u_j - u_i)/(u_i + u_j)): heating goes mostly
  //   to the particle with the lower specific energy, cooling is drawn mostly
  //   from the one with the higher (1/2 when u_i + u_j = 0 or E_ij = 0).
  void calcRates(int64_t i, T dv[3], T& du) {
    ensureRho(i);
    const auto& nb = unionset(i);
    T acc[3] = {T(0.0), T(0.0), T(0.0)};
    T eacc(0.0);
    for (int64_t j : nb) {
      if (wind(i) || wind(j)) continue;  // winds feel and exert no hydro force
      ensureRho(j);
      T xij[3], xji[3];
      sep(i, j, xij);
      for (int a = 0; a < 3; ++a) xji[a] = T(0.0) - xij[a];
      bool rk = !(flag[i] || flag[j]);
      T WRi, Gi[3], WRj, Gj[3];
      corrected(i, xij, false, rk, WRi, Gi);
      corrected(j, xji, false, rk, WRj, Gj);
      T vij[3] = {v[0][i] - v[0][j], v[1][i] - v[1][j], v[2][i] - v[2][j]};
      // artificial viscosity with the velocity-gradient limiter
      T gvi_x[3], gvj_x[3];
      for (int a = 0; a < 3; ++a) {
        gvi_x[a] = gradv[i][a * 3 + 0] * xij[0] + gradv[i][a * 3 + 1] * xij[1] + gradv[i][a * 3 + 2] * xij[2];
        gvj_x[a] = gradv[j][a * 3 + 0] * xij[0] + gradv[j][a * 3 + 1] * xij[1] + gradv[j][a * 3 + 2] * xij[2];
      }
      T phi(0.0);
      if (p.limiter) {
        T an = dot3(xij, gvi_x);
        T bd = dot3(xij, gvj_x);
        T rr = (val(bd) == 0.0) ? T(0.0) : an / bd;
        T opr = T(1.0) + rr;
        phi = tmax(T(0.0), tmin(T(1.0), T(4.0) * rr / (opr * opr)));
        T r = sqrt(dot3(xij, xij));
        T eta_m = tmin(r / h[i], r / h[j]);
        if (val(eta_m) < p.eta_crit) {
          T z = (eta_m - T(p.eta_crit)) / T(p.eta_fold);
          phi = phi * exp(T(0.0) - z * z);
        }
      }
      T vhat[3];
      for (int a = 0; a < 3; ++a) vhat[a] = vij[a] - T(0.5) * phi * (gvi_x[a] + gvj_x[a]);
      T etai[3] = {xij[0] / h[i], xij[1] / h[i], xij[2] / h[i]};
      T etaj[3] = {xij[0] / h[j], xij[1] / h[j], xij[2] / h[j]};
      T mui = tmin(T(0.0), dot3(vhat, etai) / (dot3(etai, etai) + T(p.eps2)));
      T muj = tmin(T(0.0), dot3(vhat, etaj) / (dot3(etaj, etaj) + T(p.eps2)));
      T Qi = rho[i] * (T(0.0) - T(p.Cl) * cs[i] * mui + T(p.Cq) * mui * mui);
      T Qj = rho[j] * (T(0.0) - T(p.Cl) * cs[j] * muj + T(p.Cq) * muj * muj);
      T F[3];
      if (p.q_side) {
        T VV = T(-0.5) * V[i] * V[j];
        T PP = P[i] + P[j];
        for (int a = 0; a < 3; ++a)
          F[a] = VV * (PP * (Gi[a] - Gj[a]) + T(2.0) * (Qi * Gi[a] - Qj * Gj[a]));
      } else {
        T Pi = P[i] + P[j] + Qi + Qj;
        T pre = T(-0.5) * V[i] * V[j] * Pi;
        for (int a = 0; a < 3; ++a) F[a] = pre * (Gi[a] - Gj[a]);
      }
      for (int a = 0; a < 3; ++a) acc[a] += F[a] / m[i];
      T w = F[0] * (v[0][j] - v[0][i]) + F[1] * (v[1][j] - v[1][i]) + F[2] * (v[2][j] - v[2][i]);
      T f(0.5);
      if (p.energy_split) {
        double su = val(u[i]) + val(u[j]);
        double sg = val(w) > 0 ? 1.0 : (val(w) < 0 ? -1.0 : 0.0);
        if (su > 0 && sg != 0) f = T(0.5) * (T(1.0) + T(sg) * (u[j] - u[i]) / (u[i] + u[j]));
      }
      eacc += f * w;
    }
    for (int a = 0; a < 3; ++a) dv[a] = acc[a];
    du = eacc / m[i];
  }

  // reproduction diagnostics of the corrected kernel at particle i
  void diag(int64_t i, double out[16], double tout[16]) {
    ensureMom(i);
    const auto& nb = gather(i);
    T s0(0.0), s1[3], g0[3], g1[9];
    for (int a = 0; a < 3; ++a) { s1[a] = T(0.0); g0[a] = T(0.0); }
    for (int k = 0; k < 9; ++k) g1[k] = T(0.0);
    for (int64_t j : nb) {
      ensureV(j);
      T xij[3];
      sep(i, j, xij);
      T WR, Gr[3];
      corrected(i, xij, j == i, true, WR, Gr);
      s0 += V[j] * WR;
      for (int a = 0; a < 3; ++a) s1[a] += V[j] * WR * xij[a];
      for (int a = 0; a < 3; ++a) g0[a] += V[j] * Gr[a];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) g1[a * 3 + b] += V[j] * xij[a] * Gr[b];
    }
    T all[16];
    all[0] = s0;
    for (int a = 0; a < 3; ++a) { all[1 + a] = s1[a]; all[4 + a] = g0[a]; }
    for (int k = 0; k < 9; ++k) all[7 + k] = g1[k];
    for (int k = 0; k < 16; ++k) { out[k] = val(all[k]); if (tout) tout[k] = tan_of(all[k]); }
  }
};

int check_inputs(int64_t n, const double* x, const double* h, const double* m,
                 const double* v, const double* u, double L) {
  if (n < 0 || !(L > 0) || !std::isfinite(L)) return EINVAL_;
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      double xa = x[a * n + i];
      if (!std::isfinite(xa)) return ENONFINITE_;
      if (xa < 0 || xa >= L) return EDOMAIN_;
      if (v && !std::isfinite(v[a * n + i])) return ENONFINITE_;
    }
    if (!std::isfinite(h[i]) || (m && !std::isfinite(m[i])) || (u && !std::isfinite(u[i])))
      return ENONFINITE_;
    if (!(h[i] > 0) || !(h[i] < 0.5 * L)) return EDOMAIN_;
    if (m && !(m[i] > 0)) return EINVAL_;
    if (u && !(u[i] >= 0)) return EINVAL_;
  }
  return OK;
}

template <class T>
void load_inputs(Eval<T>& E, const double* x, const double* h, const double* m, const double* v,
                 const double* u, const double* tx, const double* th, const double* tv,
                 const double* tu);

template <>
void load_inputs<double>(Eval<double>& E, const double* x, const double* h, const double* m,
                         const double* v, const double* u, const double*, const double*,
                         const double*, const double*) {
  int64_t n = E.n;
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      E.x[a][i] = x[a * n + i];
      E.v[a][i] = v ? v[a * n + i] : 0.0;
    }
    E.h[i] = h[i];
    E.m[i] = m[i];
    E.u[i] = u ? u[i] : 0.0;
  }
}
template <>
void load_inputs<Dual>(Eval<Dual>& E, const double* x, const double* h, const double* m,
                       const double* v, const double* u, const double* tx, const double* th,
                       const double* tv, const double* tu) {
  int64_t n = E.n;
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      E.x[a][i] = Dual(x[a * n + i], tx ? tx[a * n + i] : 0.0);
      E.v[a][i] = Dual(v ? v[a * n + i] : 0.0, tv ? tv[a * n + i] : 0.0);
    }
    E.h[i] = Dual(h[i], th ? th[i] : 0.0);
    E.m[i] = Dual(m[i], 0.0);
    E.u[i] = Dual(u ? u[i] : 0.0, tu ? tu[i] : 0.0);
  }
}

template <>
void load_inputs<Cnt>(Eval<Cnt>& E, const double* x, const double* h, const double* m,
                      const double* v, const double* u, const double*, const double*,
                      const double*, const double*) {
  int64_t n = E.n;
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      E.x[a][i] = Cnt(x[a * n + i]);
      E.v[a][i] = Cnt(v ? v[a * n + i] : 0.0);
    }
    E.h[i] = Cnt(h[i]);
    E.m[i] = Cnt(m[i]);
    E.u[i] = Cnt(u ? u[i] : 0.0);
  }
}
template <>
void load_inputs<CDual>(Eval<CDual>& E, const double* x, const double* h, const double* m,
                        const double* v, const double* u, const double* tx, const double* th,
                        const double* tv, const double* tu) {
  int64_t n = E.n;
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      E.x[a][i] = CDual(x[a * n + i], tx ? tx[a * n + i] : 0.0);
      E.v[a][i] = CDual(v ? v[a * n + i] : 0.0, tv ? tv[a * n + i] : 0.0);
    }
    E.h[i] = CDual(h[i], th ? th[i] : 0.0);
    E.m[i] = CDual(m[i], 0.0);
    E.u[i] = CDual(u ? u[i] : 0.0, tu ? tu[i] : 0.0);
  }
}

template <class T>
int run(int64_t n, const double* x, const double* h, const double* m, const double* v,
        const double* u, double L, const oracle_params* p, const double* tx, const double* th,
        const double* tv, const double* tu, int64_t nt, const int64_t* targets, int32_t stages,
        int32_t nthreads, int32_t use_tree, oracle_out* out, oracle_out* tout,
        const uint8_t* species = nullptr, double* Vgw_out = nullptr) {
  int rc = check_inputs(n, x, h, m, v, u, L);
  if (rc) return rc;
  if (nt < 0 || stages < 1 || stages > 4 || !p) return EINVAL_;
  for (int64_t k = 0; k < nt; ++k)
    if (targets && (targets[k] < 0 || targets[k] >= n)) return EINVAL_;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  Box box{n, x, h, L};
  KDTree* tree = use_tree ? new KDTree(&box) : nullptr;
  Eval<T> E(box, tree, *p);
  load_inputs<T>(E, x, h, m, v, u, tx, th, tv, tu);
  if (species) E.sp.assign(species, species + n);
  const bool all = (targets == nullptr);
  if (all) {
    // Whole-box evaluation: run each stage for every particle, in stage order,
    // so the memoised values a stage reads are complete before it starts.
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) { E.gather(i); E.calcV(i); }
    if (stages >= 2) {
#pragma omp parallel for schedule(dynamic, 64)
      for (int64_t i = 0; i < n; ++i) E.calcMom(i);
    }
    if (stages >= 3) {
#pragma omp parallel for schedule(dynamic, 64)
      for (int64_t i = 0; i < n; ++i) E.calcRho(i);
    }
  }
  // outputs; in target mode the stages are computed lazily and memoised
  std::vector<T> dv3(3 * nt), du(nt);
  auto emit = [&](int64_t k) {
    int64_t i = all ? k : targets[k];
    E.ensureV(i);
    if (out && out->kgather) out->kgather[k] = (int64_t)E.gather(i).size() - 1;
    if (out && out->kunion) out->kunion[k] = (int64_t)E.unionset(i).size();
    if (stages >= 2) E.ensureMom(i);
    if (stages >= 3) E.ensureRho(i);
    if (stages >= 4) {
      T d[3], e;
      E.calcRates(i, d, e);
      for (int a = 0; a < 3; ++a) dv3[a * nt + k] = d[a];
      du[k] = e;
    }
  };
  if (all) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < nt; ++k) emit(k);
  } else {
    for (int64_t k = 0; k < nt; ++k) emit(k);
  }
  int64_t nsing = 0;
  for (int64_t i = 0; i < n; ++i) nsing += E.sing[i];
  for (int side = 0; side < 2; ++side) {
    oracle_out* o = side == 0 ? out : tout;
    if (!o) continue;
    auto pick = [side](const T& a) { return side == 0 ? val(a) : tan_of(a); };
    for (int64_t k = 0; k < nt; ++k) {
      int64_t i = all ? k : targets[k];
      if (o->V) o->V[k] = pick(E.V[i]);
      if (side == 0 && Vgw_out) Vgw_out[k] = val(E.Vgw[i]);
      if (stages >= 2) {
        if (o->coef) for (int c = 0; c < 16; ++c) o->coef[c * nt + k] = pick(E.coef[i][c]);
        if (o->mom) for (int c = 0; c < 40; ++c) o->mom[c * nt + k] = pick(E.mom[i][c]);
        if (o->diag) {
          double dd[16], td[16];
          E.diag(i, dd, td);
          for (int c = 0; c < 16; ++c) o->diag[c * nt + k] = side == 0 ? dd[c] : td[c];
        }
      }
      if (stages >= 3) {
        if (o->rho) o->rho[k] = pick(E.rho[i]);
        if (o->gradv) for (int c = 0; c < 9; ++c) o->gradv[c * nt + k] = pick(E.gradv[i][c]);
        if (o->P) o->P[k] = pick(E.P[i]);
        if (o->cs) o->cs[k] = pick(E.cs[i]);
        if (o->flag) o->flag[k] = E.flag[i];
      }
      if (stages >= 4) {
        if (o->dvdt) for (int a = 0; a < 3; ++a) o->dvdt[a * nt + k] = pick(dv3[a * nt + k]);
        if (o->dudt) o->dudt[k] = pick(du[k]);
      }
    }
    if (o->nsingular) *o->nsingular = nsing;
  }
  delete tree;
  return nsing > 0 ? ESINGULAR_ : OK;
}

// Active-set evaluation (App. A.1: passive particles reuse the correction
// coefficients of their last active step; the power-of-two time bins of Sec. 2
// decide which particles are active).  flags[i] bit 0: active (density,
// velocity gradient and rates are evaluated); bit 1: volume and coefficients
// are recomputed (implied by bit 0).  Every other per-particle field is taken
// from the given state: V and coefficients for particles without bit 0 or 1,
// density and velocity gradient for particles without bit 0 (their pressure,
// sound speed and relaxation flag follow from that density, u and the
// velocity gradient as for a fresh one).  Stage by stage over the particles
// that recompute it, so every memoised value a stage reads is complete.
// Outputs (all optional, caller order, length n): V, coef, rho, gradv for every
// particle (fresh or state), dvdt, dudt for active particles (0 elsewhere).
int run_state(int64_t n, const double* x, const double* h, const double* m, const double* v,
              const double* u, double L, const oracle_params* p, const uint8_t* flags,
              const double* V_state, const double* coef_state, const double* rho_state,
              const double* gradv_state, int32_t nthreads, oracle_out* out) {
  int rc = check_inputs(n, x, h, m, v, u, L);
  if (rc) return rc;
  if (!p || !flags || !V_state || !coef_state || !rho_state || !gradv_state) return EINVAL_;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  Box box{n, x, h, L};
  KDTree tree(&box);
  Eval<double> E(box, &tree, *p);
  load_inputs<double>(E, x, h, m, v, u, nullptr, nullptr, nullptr, nullptr);
  auto active = [flags](int64_t i) { return (flags[i] & 1) != 0; };
  auto recompute = [flags](int64_t i) { return (flags[i] & 3) != 0; };
  for (int64_t i = 0; i < n; ++i) {
    if (!recompute(i)) {
      E.V[i] = V_state[i];
      E.Vgw[i] = V_state[i];  // all gas in the active-set evaluation
      E.doneV[i] = 1;
      for (int c = 0; c < 16; ++c) E.coef[i][c] = coef_state[c * n + i];
      E.doneM[i] = 1;
    }
    if (!active(i)) {
      E.rho[i] = rho_state[i];
      for (int c = 0; c < 9; ++c) E.gradv[i][c] = gradv_state[c * n + i];
      E.P[i] = (p->gamma - 1.0) * E.rho[i] * E.u[i];
      E.cs[i] = std::sqrt(p->gamma * (p->gamma - 1.0) * E.u[i]);
      double div = E.gradv[i][0] + E.gradv[i][4] + E.gradv[i][8];
      E.flag[i] = (p->relax_dt > 0 && std::exp(std::fabs(div) * p->relax_dt) > 8.0) ? 1 : 0;
      E.doneR[i] = 1;
    }
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) { E.gather(i); E.unionset(i); if (recompute(i)) E.calcV(i); }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) if (recompute(i)) E.calcMom(i);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) if (active(i)) E.calcRho(i);
  std::vector<double> dv3(3 * n, 0.0), du(n, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    if (!active(i)) continue;
    double d[3], e;
    E.calcRates(i, d, e);
    for (int a = 0; a < 3; ++a) dv3[a * n + i] = d[a];
    du[i] = e;
  }
  int64_t nsing = 0;
  for (int64_t i = 0; i < n; ++i) nsing += recompute(i) ? E.sing[i] : 0;
  if (out) {
    for (int64_t i = 0; i < n; ++i) {
      if (out->V) out->V[i] = E.V[i];
      if (out->coef) for (int c = 0; c < 16; ++c) out->coef[c * n + i] = E.coef[i][c];
      if (out->rho) out->rho[i] = E.rho[i];
      if (out->gradv) for (int c = 0; c < 9; ++c) out->gradv[c * n + i] = E.gradv[i][c];
      if (out->P) out->P[i] = E.P[i];
      if (out->cs) out->cs[i] = E.cs[i];
      if (out->flag) out->flag[i] = E.flag[i];
      if (out->dvdt) for (int a = 0; a < 3; ++a) out->dvdt[a * n + i] = dv3[a * n + i];
      if (out->dudt) out->dudt[i] = du[i];
    }
    if (out->nsingular) *out->nsingular = nsing;
  }
  return nsing > 0 ? ESINGULAR_ : OK;
}

}  // namespace

extern "C" {

// Neighbor sets as CSR.  mode 0: gather set G(i) (self included); mode 1:
// union set U(i).  method 0: brute force; method 1: k-d tree.  Columns of each
// row are sorted.  Returns 1 (EINVAL) if the capacity is too small (nnz is
// still set to the required size).
int oracle_neighbors(int32_t mode, int32_t method, int64_t n, const double* x, const double* h,
                     double L, int64_t* row_ptr, int32_t* col, int64_t cap, int64_t* nnz) {
  int rc = check_inputs(n, x, h, nullptr, nullptr, nullptr, L);
  if (rc) return rc;
  Box box{n, x, h, L};
  KDTree* tree = method ? new KDTree(&box) : nullptr;
  std::vector<std::vector<int64_t>> rows(n);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    auto pred = [&box, mode](int64_t a, int64_t c) {
      return mode == 0 ? box.in_gather(a, c) : box.in_union(a, c);
    };
    if (tree) tree->query(i, mode == 1, pred, rows[i]);
    else for (int64_t j = 0; j < n; ++j) if (pred(i, j)) rows[i].push_back(j);
  }
  delete tree;
  int64_t tot = 0;
  row_ptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) { tot += (int64_t)rows[i].size(); row_ptr[i + 1] = tot; }
  *nnz = tot;
  if (tot > cap) return EINVAL_;
  for (int64_t i = 0; i < n; ++i)
    for (size_t k = 0; k < rows[i].size(); ++k) col[row_ptr[i] + (int64_t)k] = (int32_t)rows[i][k];
  return OK;
}

// Pair counts of the whole box without storing the sets: the ordered gather
// pairs (j in G(i), j != i) and union pairs (j in U(i)), each particle's union
// set found by the k-d tree and every member tested with the gather
// predicate, so the counts equal the sizes of oracle_neighbors' sets.
int oracle_count_pairs(int64_t n, const double* x, const double* h, double L, int64_t* gather,
                       int64_t* union_) {
  int rc = check_inputs(n, x, h, nullptr, nullptr, nullptr, L);
  if (rc) return rc;
  Box box{n, x, h, L};
  KDTree tree(&box);
  int64_t g = 0, u = 0;
#pragma omp parallel reduction(+ : g, u)
  {
    std::vector<int64_t> row;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      row.clear();
      tree.query(i, true, [&box](int64_t a, int64_t c) { return box.in_union(a, c); }, row);
      u += (int64_t)row.size();
      for (int64_t j : row) g += box.in_gather(i, j) ? 1 : 0;
    }
  }
  *gather = g;
  *union_ = u;
  return OK;
}

// Forward evaluation.  targets == NULL evaluates every particle (OpenMP over
// particles); otherwise only the listed particles, computing the needed
// neighbor closure lazily on one thread.  stages: 1 volume, 2 + coefficients,
// 3 + density/velocity gradient/EOS/flag, 4 + rates.
int oracle_forward(int64_t n, const double* x, const double* h, const double* m, const double* v,
                   const double* u, double L, const oracle_params* p, int64_t nt,
                   const int64_t* targets, int32_t stages, int32_t nthreads, int32_t use_tree,
                   oracle_out* out) {
  if (!targets) nt = n;
  return run<double>(n, x, h, m, v, u, L, p, nullptr, nullptr, nullptr, nullptr, nt, targets,
                     stages, nthreads, use_tree, out, nullptr);
}

// Forward evaluation with species (0 gas, 1 wind): winds enter the density
// (Eq. rhow, with the volume over gas and wind, returned in Vgw_out when
// given) and no other sum.  Otherwise as oracle_forward.
int oracle_forward_species(int64_t n, const double* x, const double* h, const double* m,
                           const double* v, const double* u, double L, const oracle_params* p,
                           const uint8_t* species, int64_t nt, const int64_t* targets,
                           int32_t stages, int32_t nthreads, int32_t use_tree, oracle_out* out,
                           double* Vgw_out) {
  if (!targets) nt = n;
  return run<double>(n, x, h, m, v, u, L, p, nullptr, nullptr, nullptr, nullptr, nt, targets,
                     stages, nthreads, use_tree, out, nullptr, species, Vgw_out);
}

// Jacobian-vector product by forward-mode dual numbers: the tangent of every
// output along the input direction (tx, tv, tu, th); any tangent may be NULL
// (zero).  Neighbor sets, image shifts, relaxation flags and the limiter's
// branches are those of the primal point.
int oracle_jvp(int64_t n, const double* x, const double* h, const double* m, const double* v,
               const double* u, double L, const oracle_params* p, const double* tx,
               const double* tv, const double* tu, const double* th, int64_t nt,
               const int64_t* targets, int32_t stages, int32_t nthreads, int32_t use_tree,
               oracle_out* out, oracle_out* tout) {
  if (!targets) nt = n;
  return run<Dual>(n, x, h, m, v, u, L, p, tx, th, tv, tu, nt, targets, stages, nthreads,
                   use_tree, out, tout);
}

// Active-set evaluation; see run_state.
int oracle_forward_state(int64_t n, const double* x, const double* h, const double* m,
                         const double* v, const double* u, double L, const oracle_params* p,
                         const uint8_t* flags, const double* V_state, const double* coef_state,
                         const double* rho_state, const double* gradv_state, int32_t nthreads,
                         oracle_out* out) {
  return run_state(n, x, h, m, v, u, L, p, flags, V_state, coef_state, rho_state, gradv_state,
                   nthreads, out);
}

// Operation counts of a whole-box evaluation up to `stages` (1 volume, 2 +
// coefficients, 3 + density and velocity gradient, 4 + rates) on one thread:
// with derivative = 0 the plain evaluation (ops[0]: its operations), with
// derivative = 1 the forward-mode derivative along (tx, tv, tu, th) (ops[0]:
// operations on values, ops[1]: operations on tangents).  The differences
// between consecutive stages, per pair of the stage's neighbor sets, are the
// algorithmic flops per pair of the matching sweeps.
int oracle_count_ops(int64_t n, const double* x, const double* h, const double* m,
                     const double* v, const double* u, double L, const oracle_params* p,
                     const double* tx, const double* tv, const double* tu, const double* th,
                     int32_t stages, int32_t derivative, int64_t* ops) {
  if (!ops) return EINVAL_;
#ifdef _OPENMP
  const int threads_before = omp_get_max_threads();
#endif
  g_val_ops = 0;
  g_tan_ops = 0;
  int rc;
  if (derivative)
    rc = run<CDual>(n, x, h, m, v, u, L, p, tx, th, tv, tu, n, nullptr, stages, 1, 1, nullptr,
                    nullptr);
  else
    rc = run<Cnt>(n, x, h, m, v, u, L, p, nullptr, nullptr, nullptr, nullptr, n, nullptr, stages,
                  1, 1, nullptr, nullptr);
  ops[0] = g_val_ops;
  ops[1] = g_tan_ops;
#ifdef _OPENMP
  omp_set_num_threads(threads_before);
#endif
  return rc;
}

// The kernel itself, for the quadrature and finite-difference pins.
void oracle_kernel(int64_t n, const double* r, double h, double* W, double* dWdr, double* g) {
  for (int64_t k = 0; k < n; ++k) {
    if (W) W[k] = kernel_W<double>(r[k], h);
    if (dWdr) dWdr[k] = kernel_dWdr<double>(r[k], h);
    if (g) g[k] = kernel_g<double>(r[k], h);
  }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
