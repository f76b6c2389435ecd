// FP64 CPU oracle of the smoothed, differentiable 2D image-method objective
// (Eertmans, Jacques, Oestges, "Fully Differentiable Ray Tracing via
// Discontinuity Smoothing for Radio Network Optimization").
//
// TEST INFRASTRUCTURE ONLY.  Plain, slow and written to be read against the
// paper: no blocking, no fusion, no reordering.  It shares no code, header or
// constant with the CUDA library; only tests/, the smoke check and the CPU
// baseline of the benchmark load it.
//
// What it computes, per receiver r and per path candidate (Sec. V):
//   1. wall frame: e = B - A, l = |e|, u = e / l, n = (-u_y, u_x);
//      d_w(p) = n . (p - A)   (signed distance to the wall's infinite line)
//      t_w(p) = u . (p - A)   (coordinate along the wall)
//   2. candidates: every wall sequence (w_1..w_k), k = 0..K, with no wall
//      repeated twice in a row (the visibility matrix of Sec. V with all
//      pairs visible except a wall with itself); ordered by k, then
//      lexicographically.
//   3. image method (Sec. V-B, item 1): I_0 = TX, I_j = I_{j-1} - 2 d_{w_j}(I_{j-1}) n_{w_j};
//      backtrace on the relaxed (infinite) walls: Q_{k+1} = RX and, for
//      j = k..1, Q_j = the intersection of the line (Q_{j+1}, I_j) with the
//      line of w_j; Q_0 = TX.
//   4. continuous validity (Sec. V-A), every comparison x0 > x1 replaced by
//      s(x0 - x1; alpha):
//        on-segment   s(t_j) s(l_j - t_j)
//        same side    s(p) s(q) + s(-p) s(-q), p = d_{w_j}(Q_{j-1}), q = d_{w_j}(Q_{j+1})
//      and obstruction of each leg Q_j -> Q_{j+1} by every wall w other than
//      the walls its two end points lie on: with X(x, y) = s(x) s(-y) + s(-x) s(y)
//      ("x and y on opposite sides"),
//        blocked = X(d_w(Q_j), d_w(Q_{j+1})) * X(m . (A_w - Q_j), m . (B_w - Q_j)),
//      m the unit normal of the leg; the leg's visibility is prod_w (1 - blocked).
//      For the sigmoid, where blocked can lie within rounding of 1 (a wall that
//      blocks a leg at large alpha), 1 - blocked is evaluated as the equal sum
//      (1 - X1) + X1 (1 - X2) with 1 - X(x, y) = s(x) s(y) + s(-x) s(-y)
//      (s(z) + s(-z) = 1): non-negative terms, no cancellation.
//   5. path power (reading of Eq. 7 as incoherent scalar power):
//        p = Gamma^k * prod_j V_j * prod_j vis_j / L^2,  L = sum of leg lengths;
//      received power P_r = sum of p over the candidates (Eq. 7's sum over S).
//   6. smoothing s (Sec. IV): unit step (Eq. 1), sigmoid (Eq. 4) or hard
//      sigmoid (Eqs. 5-6), each scaled as s(alpha x) (Eq. 3).
//
// Degenerate relaxed geometry (the line (Q_{j+1}, I_j) parallel to the wall,
// or a leg of zero length) contributes 0.
//
// Derivatives come from the scalar type: the same templated code runs with
// double (values), a forward-mode dual number, or std::complex<double>
// (complex-step differentiation, comparisons taken on the real part).

#include <cfloat>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- scalars
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(double a, Dual b) { return Dual(a) + b; }
inline Dual operator+(Dual a, double b) { return a + Dual(b); }
inline Dual operator-(double a, Dual b) { return Dual(a) - b; }
inline Dual operator-(Dual a, double b) { return a - Dual(b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator/(double a, Dual b) { return Dual(a) / b; }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, a.d * e); }
inline Dual sqrt(Dual a) { double r = std::sqrt(a.v); return Dual(r, a.d / (2.0 * r)); }
inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
inline Dual& operator*=(Dual& a, Dual b) { return a = a * b; }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -a.d * std::sin(a.v)); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), a.d * std::cos(a.v)); }

typedef std::complex<double> Cplx;

inline double re(double x) { return x; }
inline double re(const Dual& x) { return x.v; }
inline double re(const Cplx& x) { return x.real(); }

using std::cos;
using std::exp;
using std::sin;
using std::sqrt;

// ---------------------------------------------------------------- smoothing
enum Kind { SIGMOID = 0, HARD_SIGMOID = 1, STEP = 2 };

// s(x; alpha) = s(alpha x) (Eq. 3).
template <class T>
T smooth(const T& x, double alpha, int kind) {
  if (kind == STEP) {
    // Eq. 1: theta(x) = 1 if x > 0 else 0.
    return T(re(x) > 0.0 ? 1.0 : 0.0);
  }
  T z = alpha * x;
  if (kind == SIGMOID) {
    // Eq. 4: 1 / (1 + exp(-z)); the two algebraically equal forms keep the
    // exponential's argument non-positive.
    if (re(z) >= 0.0) return 1.0 / (1.0 + exp(-z));
    T e = exp(z);
    return e / (1.0 + e);
  }
  // Eqs. 5-6: relu6(z + 3) / 6 with relu6(y) = min(max(0, y), 6).
  T y = z + 3.0;
  if (re(y) <= 0.0) return T(0.0);
  if (re(y) >= 6.0) return T(1.0);
  return y / 6.0;
}

// ---------------------------------------------------------------- geometry
template <class T>
struct Vec {
  T x, y;
};
template <class T>
Vec<T> sub(const Vec<T>& a, const Vec<T>& b) { return Vec<T>{a.x - b.x, a.y - b.y}; }
template <class T>
T dot(const Vec<T>& a, const Vec<T>& b) { return a.x * b.x + a.y * b.y; }

template <class T>
struct Wall {
  Vec<T> a, b;   // end points A, B
  Vec<T> u, n;   // unit direction and unit normal of the line
  T len;         // |B - A|
};

template <class T>
Wall<T> make_wall(const T* xy) {
  Wall<T> w;
  w.a = Vec<T>{xy[0], xy[1]};
  w.b = Vec<T>{xy[2], xy[3]};
  Vec<T> e = sub(w.b, w.a);
  w.len = sqrt(dot(e, e));
  w.u = Vec<T>{e.x / w.len, e.y / w.len};
  w.n = Vec<T>{-w.u.y, w.u.x};
  return w;
}

// signed distance of p to the wall's line
template <class T>
T dist_line(const Wall<T>& w, const Vec<T>& p) { return dot(w.n, sub(p, w.a)); }

// coordinate of p along the wall, from A towards B
template <class T>
T along(const Wall<T>& w, const Vec<T>& p) { return dot(w.u, sub(p, w.a)); }

// mirror image of p across the wall's line
template <class T>
Vec<T> mirror(const Wall<T>& w, const Vec<T>& p) {
  T d = dist_line(w, p);
  return Vec<T>{p.x - 2.0 * d * w.n.x, p.y - 2.0 * d * w.n.y};
}

// ---------------------------------------------------------------- candidates
// All sequences of 0..K walls with no immediate repeat; by length, then
// lexicographic.
std::vector<std::vector<int>> candidates(int W, int K) {
  std::vector<std::vector<int>> out;
  out.push_back(std::vector<int>());
  std::vector<std::vector<int>> level(1);
  for (int k = 1; k <= K; ++k) {
    std::vector<std::vector<int>> next;
    for (const auto& s : level)
      for (int w = 0; w < W; ++w) {
        if (!s.empty() && s.back() == w) continue;
        std::vector<int> t = s;
        t.push_back(w);
        next.push_back(t);
      }
    for (const auto& s : next) out.push_back(s);
    level.swap(next);
  }
  return out;
}

struct Params {
  int K;
  double alpha;
  int kind;
  double gamma;
};

// Per-path record for inspection by tests (filled only when requested).
struct PathRecord {
  int degenerate;
  double verts[2 * 8];   // up to K = 6: Q_0..Q_{k+1}
  double validity;       // prod_j V_j
  double vis[7];         // per-leg visibility
  double length;         // L
  double power;          // p
};

// Visibility of every leg of the path Q_0..Q_{k+1} (its unit normals in
// leg_normal): each leg Q_j -> Q_{j+1} is tested against every wall other than
// the walls its two end points lie on; returns the product over the legs.
template <class T>
T obstruction(const std::vector<Wall<T>>& walls, const std::vector<Vec<T>>& Q,
              const std::vector<Vec<T>>& leg_normal, const std::vector<int>& seq,
              const Params& P, PathRecord* rec) {
  const int k = (int)seq.size();
  const int W = (int)walls.size();
  const double a = P.alpha;
  const int kind = P.kind;
  T visibility = T(1.0);
  for (int j = 0; j <= k; ++j) {
    const int skip_a = (j >= 1) ? seq[j - 1] : -1;     // wall holding Q_j
    const int skip_b = (j + 1 <= k) ? seq[j] : -1;     // wall holding Q_{j+1}
    T vis = T(1.0);
    for (int wi = 0; wi < W; ++wi) {
      if (wi == skip_a || wi == skip_b) continue;
      const Wall<T>& w = walls[wi];
      // the leg's end points on opposite sides of the wall's line ...
      T x1 = dist_line(w, Q[j]);
      T y1 = dist_line(w, Q[j + 1]);
      T cross1 = smooth(x1, a, kind) * smooth(T(-y1), a, kind) +
                 smooth(T(-x1), a, kind) * smooth(y1, a, kind);
      // ... and the wall's end points on opposite sides of the leg's line
      T x2 = dot(leg_normal[j], sub(w.a, Q[j]));
      T y2 = dot(leg_normal[j], sub(w.b, Q[j]));
      T cross2 = smooth(x2, a, kind) * smooth(T(-y2), a, kind) +
                 smooth(T(-x2), a, kind) * smooth(y2, a, kind);
      if (kind == SIGMOID) {
        // 1 - cross1 cross2 = (1 - cross1) + cross1 (1 - cross2), each complement
        // "both on one side" written out
        T same1 = smooth(x1, a, kind) * smooth(y1, a, kind) +
                  smooth(T(-x1), a, kind) * smooth(T(-y1), a, kind);
        T same2 = smooth(x2, a, kind) * smooth(y2, a, kind) +
                  smooth(T(-x2), a, kind) * smooth(T(-y2), a, kind);
        vis = vis * (same1 + cross1 * same2);
      } else {
        vis = vis * (1.0 - cross1 * cross2);
      }
    }
    if (rec && j < 7) rec->vis[j] = re(vis);
    visibility = visibility * vis;
  }
  return visibility;
}

// Geometry, validity and visibility of one path candidate `seq` (k = seq.size()).
template <class T>
struct PathTerms {
  bool degenerate;
  T validity;                // prod_j V_j
  T visibility;              // prod_j vis_j
  T L;                       // sum of the leg lengths
  std::vector<T> cos_in;     // |cos| of the angle between leg j-1 and wall j's normal
};

template <class T>
PathTerms<T> path_terms(const std::vector<Wall<T>>& walls, const Vec<T>& tx, const Vec<T>& rx,
                        const std::vector<int>& seq, const Params& P, PathRecord* rec) {
  PathTerms<T> out;
  out.degenerate = true;
  out.validity = out.visibility = out.L = T(0.0);
  const int k = (int)seq.size();
  const int W = (int)walls.size();
  // images I_0..I_k
  std::vector<Vec<T>> img(k + 1);
  img[0] = tx;
  for (int j = 1; j <= k; ++j) img[j] = mirror(walls[seq[j - 1]], img[j - 1]);
  // backtrace Q_0..Q_{k+1}
  std::vector<Vec<T>> Q(k + 2);
  Q[k + 1] = rx;
  Q[0] = tx;
  bool degenerate = false;
  for (int j = k; j >= 1; --j) {
    const Wall<T>& w = walls[seq[j - 1]];
    T a = dist_line(w, img[j]);
    T b = dist_line(w, Q[j + 1]);
    if (re(b) - re(a) == 0.0) { degenerate = true; break; }
    T t = b / (b - a);
    Q[j] = Vec<T>{Q[j + 1].x + (img[j].x - Q[j + 1].x) * t,
                  Q[j + 1].y + (img[j].y - Q[j + 1].y) * t};
  }
  std::vector<T> leg_len(k + 1);
  std::vector<Vec<T>> leg_normal(k + 1);
  if (!degenerate) {
    for (int j = 0; j <= k; ++j) {
      Vec<T> d = sub(Q[j + 1], Q[j]);
      T l = sqrt(dot(d, d));
      if (re(l) == 0.0) { degenerate = true; break; }
      leg_len[j] = l;
      leg_normal[j] = Vec<T>{-d.y / l, d.x / l};
    }
  }
  if (rec) {
    rec->degenerate = degenerate ? 1 : 0;
    for (int i = 0; i < k + 2 && i < 8; ++i) {
      rec->verts[2 * i] = degenerate ? NAN : re(Q[i].x);
      rec->verts[2 * i + 1] = degenerate ? NAN : re(Q[i].y);
    }
  }
  if (degenerate) {
    if (rec) { rec->validity = 0; rec->length = 0; rec->power = 0; }
    return out;
  }
  const double a = P.alpha;
  const int kind = P.kind;
  // continuous validity of each reflection
  T validity = T(1.0);
  for (int j = 1; j <= k; ++j) {
    const Wall<T>& w = walls[seq[j - 1]];
    T tj = along(w, Q[j]);
    T on_seg = smooth(tj, a, kind) * smooth(w.len - tj, a, kind);
    T p = dist_line(w, Q[j - 1]);
    T q = dist_line(w, Q[j + 1]);
    T same_side = smooth(p, a, kind) * smooth(q, a, kind) +
                  smooth(T(-p), a, kind) * smooth(T(-q), a, kind);
    validity = validity * on_seg * same_side;
  }
  // obstruction of each leg
  T visibility = obstruction(walls, Q, leg_normal, seq, P, rec);
  T L = T(0.0);
  for (int j = 0; j <= k; ++j) L = L + leg_len[j];
  // incidence at each reflection: the incoming leg j-1 is Q_{j-1} -> Q_j, whose unit
  // normal is leg_normal[j-1]; |u_w . m| = |n_w . d| / |d| for the leg direction d
  out.cos_in.resize(k);
  for (int j = 1; j <= k; ++j) {
    const Wall<T>& w = walls[seq[j - 1]];
    T c = dot(w.u, leg_normal[j - 1]);
    out.cos_in[j - 1] = re(c) < 0.0 ? T(-c) : c;
  }
  out.degenerate = false;
  out.validity = validity;
  out.visibility = visibility;
  out.L = L;
  if (rec) {
    rec->validity = re(validity);
    rec->length = re(L);
  }
  return out;
}

// Power of one path candidate `seq` (k = seq.size()) from tx to rx.
template <class T>
T path_power(const std::vector<Wall<T>>& walls, const Vec<T>& tx, const Vec<T>& rx,
             const std::vector<int>& seq, const Params& P, PathRecord* rec) {
  const int k = (int)seq.size();
  PathTerms<T> t = path_terms(walls, tx, rx, seq, P, rec);
  if (t.degenerate) return T(0.0);
  const T& validity = t.validity;
  const T& visibility = t.visibility;
  const T& L = t.L;
  double gk = 1.0;
  for (int j = 0; j < k; ++j) gk *= P.gamma;
  T power = gk * validity * visibility / (L * L);
  if (rec) rec->power = re(power);
  return power;
}

// Fresnel reflection coefficient for a field normal to the plane of incidence
// (TE): (c - sqrt(eps - s^2)) / (c + sqrt(eps - s^2)), with c the cosine of the
// angle of incidence, s^2 = 1 - c^2 and eps the wall's relative permittivity.  At
// eps = 1 the coefficient is 0 for every c > 0; c = 0 (grazing) keeps that value.
template <class T>
T fresnel_te(const T& c, double eps) {
  const T r = sqrt(eps - (1.0 - c * c));
  if (re(c) + re(r) == 0.0) return T(0.0);
  return (c - r) / (c + r);
}

// Eq. 7 read as a coherent sum of scalar fields (field normal to the scene plane,
// free-space spreading 1/L of the unfolded path): the field of one path is
//   prod_j C_j * V * vis * exp(-i 2 pi L / lambda) / L,
// with C_j the Fresnel TE coefficient at reflection j (eps > 0), or the constant
// amplitude -sqrt(Gamma) (eps == 0), whose square is the power coefficient Gamma.
// Returned as (re, im).
template <class T>
Vec<T> path_field(const std::vector<Wall<T>>& walls, const Vec<T>& tx, const Vec<T>& rx,
                  const std::vector<int>& seq, const Params& P, double wavelength, double eps,
                  double* length) {
  PathTerms<T> t = path_terms(walls, tx, rx, seq, P, nullptr);
  *length = t.degenerate ? 0.0 : re(t.L);
  if (t.degenerate) return Vec<T>{T(0.0), T(0.0)};
  T coef = T(1.0);
  for (const T& c : t.cos_in) coef = coef * ((eps > 0.0) ? fresnel_te(c, eps) : T(-std::sqrt(P.gamma)));
  const T amp = coef * t.validity * t.visibility / t.L;
  const T phase = (2.0 * M_PI / wavelength) * t.L;
  return Vec<T>{amp * cos(phase), -(amp * sin(phase))};
}

// ---------------------------------------------------------------- path finder
// Sec. V-B, "Continuous Path Finding": besides the image method, the framework
// finds the reflection points iteratively and checks convergence with the
// Min-Path-Tracing (MPT) cost, whose comparison with zero is smoothed by s.  The
// paper defers the formulation to the MPT paper; the reading here, for
// reflections on the walls' infinite lines, is:
//   unknowns   tau_j, the coordinate of reflection point X_j = A_j + tau_j u_j
//              along wall w_j (j = 1..k); X_0 = TX, X_{k+1} = RX;
//   legs       d_j = X_{j+1} - X_j, l_j = |d_j|, unit direction h_j = d_j / l_j;
//   residuals  r_j = h_j - R_j h_{j-1}, R_j v = v - 2 (n_j . v) n_j (the mirror of
//              wall j): zero iff the reflection law holds at X_j; the MPT cost is
//              C = sum_j |r_j|^2;
//   start      tau_j = len_j / 2 (every wall's midpoint);
//   each step  a Gauss-Newton step on the residuals, (J^T J + mu) delta = -J^T r with
//              dh_j / dX_{j+1} = -dh_j / dX_j = (I - h_j h_j^T) / l_j and mu = 1e-6
//              times the diagonal (a Levenberg term that keeps a grazing leg's
//              singular system solvable); every delta_j clamped to [-len_j, len_j]
//              (a valid point lies within len_j / 2 of the start); then
//              backtracking: the largest fraction 2^-m (m < 12) of delta that lowers
//              C by 1e-4 of its slope along delta, up to 8 units of rounding of C,
//              and no step if none does;
//   check      kappa = s(eps - C) with C at the final points;
//   validity   prod_j s(tau_j) s(len_j - tau_j) * kappa: the convergence check takes
//              the place of the image method's same-side test (a converged
//              reflection has its neighbours on one side);
//   degenerate a leg of zero length at any step, or a leg shorter than 1e-3 (in the
//              scene's length unit) at the final points: the path contributes 0
//              (iterations that run into the corner where two walls meet shrink the
//              leg between them towards zero without converging; at 1e-3 such a
//              leg is still long enough that single and double precision runs of
//              the finder agree on which side of the limit it ends);
// Fermat path tracing (FPT) takes the same unknowns, start, clamp, check, validity
// and degenerate rule, with the total path length as the objective:
//   L = sum_j l_j, dL/dtau_j = u_j . (h_{j-1} - h_j),
//   d2L/dtau_j^2 = u_j^T (I - h_{j-1} h_{j-1}^T) u_j / l_{j-1} + u_j^T (I - h_j h_j^T) u_j / l_j,
//   d2L/dtau_j dtau_{j+1} = -u_j^T (I - h_j h_j^T) u_{j+1} / l_j;
//   each step  a Newton step (H + mu) delta = -grad L (L is convex in tau: a sum of
//              norms of affine functions), clamped, with the same backtracking on L;
//   check      the MPT cost C at the final points, as for MPT (the paper checks the
//              convergence of every finder with the MPT loss).  Where the wall's
//              line separates the path's neighbours, the length's minimum is the
//              straight line through the crossing point, whose C is 4 (i . n)^2:
//              the check rejects it.
struct FinderLegs {
  std::vector<Vec<double>> X, h;   // vertices X_0..X_{k+1}; unit leg directions h_0..h_k
  std::vector<double> l;           // leg lengths
  bool degenerate;
};

FinderLegs finder_legs(const std::vector<Wall<double>>& walls, const Vec<double>& tx,
                       const Vec<double>& rx, const std::vector<int>& seq,
                       const std::vector<double>& tau) {
  const int k = (int)seq.size();
  FinderLegs f;
  f.X.resize(k + 2);
  f.h.resize(k + 1);
  f.l.resize(k + 1);
  f.degenerate = false;
  f.X[0] = tx;
  f.X[k + 1] = rx;
  for (int j = 1; j <= k; ++j) {
    const Wall<double>& w = walls[seq[j - 1]];
    f.X[j] = Vec<double>{w.a.x + tau[j - 1] * w.u.x, w.a.y + tau[j - 1] * w.u.y};
  }
  for (int j = 0; j <= k; ++j) {
    const Vec<double> d = sub(f.X[j + 1], f.X[j]);
    f.l[j] = std::sqrt(dot(d, d));
    if (f.l[j] == 0.0) {
      f.degenerate = true;
      return f;
    }
    f.h[j] = Vec<double>{d.x / f.l[j], d.y / f.l[j]};
  }
  return f;
}

constexpr int FINDER_HALVINGS = 12;
constexpr double MPT_MIN_LEG = 1e-3;

// reflection law residual r_j = h_j - R_j h_{j-1} at point j (1..k)
Vec<double> mpt_residual(const Wall<double>& w, const Vec<double>& hin, const Vec<double>& hout) {
  const double in = dot(w.n, hin);
  return Vec<double>{hout.x - (hin.x - 2.0 * in * w.n.x), hout.y - (hin.y - 2.0 * in * w.n.y)};
}

double mpt_cost(const std::vector<Wall<double>>& walls, const std::vector<int>& seq,
                const FinderLegs& f) {
  double C = 0.0;
  for (int j = 1; j <= (int)seq.size(); ++j) {
    const Vec<double> r = mpt_residual(walls[seq[j - 1]], f.h[j - 1], f.h[j]);
    C += dot(r, r);
  }
  return C;
}

// Solves the k x k symmetric positive definite system A x = b (Cholesky, in place).
void spd_solve(std::vector<double>& A, std::vector<double>& b, int k) {
  for (int c = 0; c < k; ++c) {
    double d = A[c * k + c];
    for (int p = 0; p < c; ++p) d -= A[c * k + p] * A[c * k + p];
    d = std::sqrt(d > 0.0 ? d : 0.0);
    A[c * k + c] = d;
    for (int r = c + 1; r < k; ++r) {
      double v = A[r * k + c];
      for (int p = 0; p < c; ++p) v -= A[r * k + p] * A[c * k + p];
      A[r * k + c] = d > 0.0 ? v / d : 0.0;
    }
  }
  for (int r = 0; r < k; ++r) {   // L y = b
    double v = b[r];
    for (int p = 0; p < r; ++p) v -= A[r * k + p] * b[p];
    b[r] = A[r * k + r] > 0.0 ? v / A[r * k + r] : 0.0;
  }
  for (int r = k - 1; r >= 0; --r) {   // L^T x = y
    double v = b[r];
    for (int p = r + 1; p < k; ++p) v -= A[p * k + r] * b[p];
    b[r] = A[r * k + r] > 0.0 ? v / A[r * k + r] : 0.0;
  }
}

// Reflection points of `seq` after n_iter MPT steps; returns false if the path is
// degenerate.
bool mpt_points(const std::vector<Wall<double>>& walls, const Vec<double>& tx,
                const Vec<double>& rx, const std::vector<int>& seq, int n_iter,
                std::vector<double>& tau) {
  const int k = (int)seq.size();
  tau.assign(k, 0.0);
  for (int j = 0; j < k; ++j) tau[j] = 0.5 * walls[seq[j]].len;
  if (k == 0) {
    const FinderLegs f = finder_legs(walls, tx, rx, seq, tau);
    return !f.degenerate && f.l[0] >= MPT_MIN_LEG;
  }
  auto proj = [](const FinderLegs& f, int leg, const Vec<double>& v) {   // (I - h h^T) v / l
    const double c = dot(f.h[leg], v);
    return Vec<double>{(v.x - c * f.h[leg].x) / f.l[leg], (v.y - c * f.h[leg].y) / f.l[leg]};
  };
  auto mirror_dir = [](const Wall<double>& w, const Vec<double>& v) {
    const double c = dot(w.n, v);
    return Vec<double>{v.x - 2.0 * c * w.n.x, v.y - 2.0 * c * w.n.y};
  };
  for (int it = 0; it < n_iter; ++it) {
    const FinderLegs f = finder_legs(walls, tx, rx, seq, tau);
    if (f.degenerate) return false;
    // J: entry (j, i) = dr_j / dtau_i (a 2-vector), nonzero for |i - j| <= 1
    std::vector<Vec<double>> J(k * k, Vec<double>{0.0, 0.0});
    std::vector<Vec<double>> r(k);
    for (int j = 1; j <= k; ++j) {
      const Wall<double>& w = walls[seq[j - 1]];
      r[j - 1] = mpt_residual(w, f.h[j - 1], f.h[j]);
      // tau_j moves the end of leg j - 1 and the start of leg j
      const Vec<double> a = proj(f, j, w.u), c = mirror_dir(w, proj(f, j - 1, w.u));
      J[(j - 1) * k + (j - 1)] = Vec<double>{-a.x - c.x, -a.y - c.y};
      if (j < k) J[(j - 1) * k + j] = proj(f, j, walls[seq[j]].u);   // the end of leg j
      if (j > 1)                                                     // the start of leg j - 1
        J[(j - 1) * k + (j - 2)] = mirror_dir(w, proj(f, j - 1, walls[seq[j - 2]].u));
    }
    std::vector<double> A(k * k, 0.0), b(k, 0.0);
    for (int a = 0; a < k; ++a) {
      for (int c = 0; c < k; ++c) {
        double v = 0.0;
        for (int j = 0; j < k; ++j) v += dot(J[j * k + a], J[j * k + c]);
        A[a * k + c] = v;
      }
      double v = 0.0;
      for (int j = 0; j < k; ++j) v += dot(J[j * k + a], r[j]);
      b[a] = -v;
    }
    // slope of C along the step: grad C = 2 J^T r = -2 b
    std::vector<double> g0(b);
    for (int j = 0; j < k; ++j) A[j * k + j] *= 1.0 + 1e-6;
    spd_solve(A, b, k);
    double slope = 0.0;
    for (int j = 0; j < k; ++j) {
      const double lim = walls[seq[j]].len;
      b[j] = b[j] < -lim ? -lim : (b[j] > lim ? lim : b[j]);
      slope -= 2.0 * g0[j] * b[j];
    }
    const double C0 = mpt_cost(walls, seq, f);
    const double tol = 8.0 * DBL_EPSILON * C0;
    double t = 1.0;
    for (int m = 0; m < FINDER_HALVINGS; ++m, t *= 0.5) {
      std::vector<double> trial(tau);
      for (int j = 0; j < k; ++j) trial[j] += t * b[j];
      const FinderLegs ft = finder_legs(walls, tx, rx, seq, trial);
      if (ft.degenerate) continue;
      if (mpt_cost(walls, seq, ft) <= C0 + 1e-4 * t * slope + tol) {
        tau.swap(trial);
        break;
      }
    }
  }
  const FinderLegs f = finder_legs(walls, tx, rx, seq, tau);
  if (f.degenerate) return false;
  for (double l : f.l)
    if (l < MPT_MIN_LEG) return false;
  return true;
}

// Reflection points of `seq` after n_iter Fermat (Newton) steps on the path length;
// returns false if the path is degenerate.
bool fpt_points(const std::vector<Wall<double>>& walls, const Vec<double>& tx,
                const Vec<double>& rx, const std::vector<int>& seq, int n_iter,
                std::vector<double>& tau) {
  const int k = (int)seq.size();
  tau.assign(k, 0.0);
  for (int j = 0; j < k; ++j) tau[j] = 0.5 * walls[seq[j]].len;
  auto length = [](const FinderLegs& f) {
    double L = 0.0;
    for (double l : f.l) L += l;
    return L;
  };
  // u^T (I - h h^T) v / l for leg `leg`
  auto pquad = [](const FinderLegs& f, int leg, const Vec<double>& u, const Vec<double>& v) {
    return (dot(u, v) - dot(f.h[leg], u) * dot(f.h[leg], v)) / f.l[leg];
  };
  for (int it = 0; it < n_iter && k > 0; ++it) {
    const FinderLegs f = finder_legs(walls, tx, rx, seq, tau);
    if (f.degenerate) return false;
    std::vector<double> H(k * k, 0.0), b(k, 0.0);
    for (int j = 1; j <= k; ++j) {
      const Vec<double>& u = walls[seq[j - 1]].u;
      b[j - 1] = -(dot(u, f.h[j - 1]) - dot(u, f.h[j]));   // -dL/dtau_j
      H[(j - 1) * k + (j - 1)] = pquad(f, j - 1, u, u) + pquad(f, j, u, u);
      if (j < k) {
        const double c = -pquad(f, j, u, walls[seq[j]].u);
        H[(j - 1) * k + j] = c;
        H[j * k + (j - 1)] = c;
      }
    }
    std::vector<double> g0(b);   // -grad L
    for (int j = 0; j < k; ++j) H[j * k + j] *= 1.0 + 1e-6;
    spd_solve(H, b, k);
    double slope = 0.0;
    for (int j = 0; j < k; ++j) {
      const double lim = walls[seq[j]].len;
      b[j] = b[j] < -lim ? -lim : (b[j] > lim ? lim : b[j]);
      slope -= g0[j] * b[j];
    }
    const double L0 = length(f);
    const double tol = 8.0 * DBL_EPSILON * L0;
    double t = 1.0;
    for (int m = 0; m < FINDER_HALVINGS; ++m, t *= 0.5) {
      std::vector<double> trial(tau);
      for (int j = 0; j < k; ++j) trial[j] += t * b[j];
      const FinderLegs ft = finder_legs(walls, tx, rx, seq, trial);
      if (ft.degenerate) continue;
      if (length(ft) <= L0 + 1e-4 * t * slope + tol) {
        tau.swap(trial);
        break;
      }
    }
  }
  const FinderLegs f = finder_legs(walls, tx, rx, seq, tau);
  if (f.degenerate) return false;
  for (double l : f.l)
    if (l < MPT_MIN_LEG) return false;
  return true;
}

enum Finder { FINDER_MPT = 0, FINDER_FPT = 1 };

bool finder_points(int finder, const std::vector<Wall<double>>& walls, const Vec<double>& tx,
                   const Vec<double>& rx, const std::vector<int>& seq, int n_iter,
                   std::vector<double>& tau) {
  return finder == FINDER_FPT ? fpt_points(walls, tx, rx, seq, n_iter, tau)
                              : mpt_points(walls, tx, rx, seq, n_iter, tau);
}

// Power of one path candidate whose reflection points come from a path finder
// (MPT or FPT), with the smoothed convergence check; fills tau [k], C and kappa.
double finder_path_power(int finder, const std::vector<Wall<double>>& walls,
                         const Vec<double>& tx, const Vec<double>& rx,
                         const std::vector<int>& seq, const Params& P, int n_iter, double eps,
                         std::vector<double>& tau, double* cost, double* kappa) {
  const int k = (int)seq.size();
  *cost = 0.0;
  *kappa = 0.0;
  if (!finder_points(finder, walls, tx, rx, seq, n_iter, tau)) return 0.0;
  const FinderLegs f = finder_legs(walls, tx, rx, seq, tau);
  *cost = mpt_cost(walls, seq, f);
  *kappa = smooth(eps - *cost, P.alpha, P.kind);
  double validity = *kappa;
  for (int j = 1; j <= k; ++j) {
    const Wall<double>& w = walls[seq[j - 1]];
    validity = validity * smooth(tau[j - 1], P.alpha, P.kind) *
               smooth(w.len - tau[j - 1], P.alpha, P.kind);
  }
  std::vector<Vec<double>> normal(k + 1);
  for (int j = 0; j <= k; ++j) normal[j] = Vec<double>{-f.h[j].y, f.h[j].x};
  const double visibility = obstruction(walls, f.X, normal, seq, P, nullptr);
  double L = 0.0;
  for (int j = 0; j <= k; ++j) L += f.l[j];
  double gk = 1.0;
  for (int j = 0; j < k; ++j) gk *= P.gamma;
  return gk * validity * visibility / (L * L);
}

template <class T>
std::vector<Wall<T>> make_walls(const std::vector<T>& xy, int W) {
  std::vector<Wall<T>> walls;
  walls.reserve(W);
  for (int i = 0; i < W; ++i) walls.push_back(make_wall<T>(&xy[4 * i]));
  return walls;
}

// P_r for one receiver, summed over the candidate table in order.
template <class T>
T received_power(const std::vector<Wall<T>>& walls, const Vec<T>& tx, const Vec<T>& rx,
                 const std::vector<std::vector<int>>& cands, const Params& P) {
  T sum = T(0.0);
  for (const auto& seq : cands) sum = sum + path_power(walls, tx, rx, seq, P, nullptr);
  return sum;
}

int check_args(const double* walls, int W, const double* tx, const double* rx, int R, int K,
               double alpha, int kind) {
  if (!walls || !tx || (R > 0 && !rx)) return 1;
  if (W < 1 || R < 0 || K < 0 || K > 6 || !(alpha >= 0.0)) return 1;
  if (kind < 0 || kind > 2) return 1;
  return 0;
}

void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

// ---------------------------------------------------------------- 3D scenes
// Sec. VI: the method is not tied to two dimensions.  Read for triangle walls:
//   plane of triangle (A, B, C): unit normal n along (B - A) x (C - A), offset
//   c = n . A, signed distance d(p) = n . p - c; edge k (A->B, B->C, C->A) has the
//   in-plane unit normal m_k = n x e_k / |e_k| (pointing into the triangle) and the
//   signed in-plane distance delta_k(p) = m_k . (p - start of edge k).
//   image method and backtrace: as in 2D with planes for lines;
//   on the object: prod_k s(delta_k(Q_j)) (the 2D on-segment test has two ends);
//   same side: s(p) s(q) + s(-p) s(-q) with plane distances;
//   obstruction of leg Q_j -> Q_{j+1} by triangle w (not one in the plane of a
//   triangle its end points lie on: the leg meets that plane only at the end
//   point): X(x, y) * prod_k s(delta_k(P)), x = d_w(Q_j), y = d_w(Q_{j+1}), P the
//   intersection of the leg's line with w's plane (no intersection: not blocked);
//   for the sigmoid 1 - blocked is evaluated without cancellation as in 2D;
//   path power Gamma^k V vis / L^2 as in 2D;
//   two consecutive reflections on triangles of one plane (normals parallel and
//   offsets equal to within 1e-5): a degenerate path (zero-length leg), power 0.
template <class T>
struct V3 {
  T x, y, z;
};
template <class T>
V3<T> operator+(const V3<T>& a, const V3<T>& b) { return V3<T>{a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T>
V3<T> operator-(const V3<T>& a, const V3<T>& b) { return V3<T>{a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T, class S>
V3<T> operator*(const S& s, const V3<T>& a) { return V3<T>{s * a.x, s * a.y, s * a.z}; }
template <class T>
T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T>
V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return V3<T>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T>
T norm(const V3<T>& a) { return sqrt(dot(a, a)); }

template <class T>
struct Tri {
  V3<T> v[3];   // corners A, B, C
  V3<T> n;      // unit normal
  T c;          // n . A
  V3<T> m[3];   // in-plane unit normals of the edges, pointing inside
};

template <class T>
Tri<T> make_tri(const T* p) {
  Tri<T> t;
  for (int i = 0; i < 3; ++i) t.v[i] = V3<T>{p[3 * i], p[3 * i + 1], p[3 * i + 2]};
  V3<T> nn = cross(t.v[1] - t.v[0], t.v[2] - t.v[0]);
  t.n = (1.0 / norm(nn)) * nn;
  t.c = dot(t.n, t.v[0]);
  for (int k = 0; k < 3; ++k) {
    V3<T> e = t.v[(k + 1) % 3] - t.v[k];
    t.m[k] = (1.0 / norm(e)) * cross(t.n, e);
  }
  return t;
}

template <class T>
T plane_dist(const Tri<T>& t, const V3<T>& p) { return dot(t.n, p) - t.c; }
template <class T>
T edge_dist(const Tri<T>& t, int k, const V3<T>& p) { return dot(t.m[k], p - t.v[k]); }

// prod_k s(delta_k(p)): p (on the plane) inside the triangle
template <class T>
T inside(const Tri<T>& t, const V3<T>& p, double alpha, int kind) {
  T r = T(1.0);
  for (int k = 0; k < 3; ++k) r *= smooth(edge_dist(t, k, p), alpha, kind);
  return r;
}

// 1 - inside(t, p) for the sigmoid as the equal sum of non-negative terms
// s(-d_0) + s(d_0) (s(-d_1) + s(d_1) s(-d_2)), d_k the in-plane edge distances
// (1 - abc = (1 - a) + a (1 - b) + ab (1 - c), with 1 - s(d) = s(-d)).
template <class T>
T outside(const Tri<T>& t, const V3<T>& p, double alpha, int kind) {
  const T d0 = edge_dist(t, 0, p), d1 = edge_dist(t, 1, p), d2 = edge_dist(t, 2, p);
  return smooth(T(-d0), alpha, kind) +
         smooth(d0, alpha, kind) * (smooth(T(-d1), alpha, kind) +
                                    smooth(d1, alpha, kind) * smooth(T(-d2), alpha, kind));
}

// Triangles a and b lie in one plane (normals parallel, offsets equal, to 1e-5).
template <class T>
bool coplanar(const Tri<T>& ta, const Tri<T>& tb) {
  const double nn = re(dot(ta.n, tb.n));
  return std::fabs(nn) >= 1.0 - 1e-5 && std::fabs(re(ta.c) - nn * re(tb.c)) <= 1e-5 * (1.0 + std::fabs(re(ta.c)));
}

template <class T>
T path_power3(const std::vector<Tri<T>>& tris, const V3<T>& tx, const V3<T>& rx,
              const std::vector<int>& seq, const Params& P) {
  const int k = (int)seq.size();
  const int W = (int)tris.size();
  std::vector<V3<T>> img(k + 1);
  img[0] = tx;
  for (int j = 1; j <= k; ++j) {
    const Tri<T>& t = tris[seq[j - 1]];
    img[j] = img[j - 1] - (2.0 * plane_dist(t, img[j - 1])) * t.n;
  }
  // two consecutive reflections in one plane (two triangles of one flat face): the
  // leg between them has zero length, so the path is degenerate
  for (int j = 1; j < k; ++j)
    if (coplanar(tris[seq[j - 1]], tris[seq[j]])) return T(0.0);
  std::vector<V3<T>> Q(k + 2);
  Q[0] = tx;
  Q[k + 1] = rx;
  for (int j = k; j >= 1; --j) {
    const Tri<T>& t = tris[seq[j - 1]];
    const T a = plane_dist(t, img[j]);
    const T b = plane_dist(t, Q[j + 1]);
    if (re(b) - re(a) == 0.0) return T(0.0);
    Q[j] = Q[j + 1] + (b / (b - a)) * (img[j] - Q[j + 1]);
  }
  T L = T(0.0);
  for (int j = 0; j <= k; ++j) {
    const T l = norm(Q[j + 1] - Q[j]);
    if (re(l) == 0.0) return T(0.0);
    L += l;
  }
  const double al = P.alpha;
  const int kind = P.kind;
  T validity = T(1.0);
  for (int j = 1; j <= k; ++j) {
    const Tri<T>& t = tris[seq[j - 1]];
    const T p = plane_dist(t, Q[j - 1]), q = plane_dist(t, Q[j + 1]);
    const T same_side = smooth(p, al, kind) * smooth(q, al, kind) +
                        smooth(-p, al, kind) * smooth(-q, al, kind);
    validity *= inside(t, Q[j], al, kind) * same_side;
  }
  // a leg meets the plane of an end point's triangle only at that end point: it is
  // not tested against any triangle of that plane
  T visibility = T(1.0);
  for (int j = 0; j <= k; ++j) {
    for (int wi = 0; wi < W; ++wi) {
      const Tri<T>& t = tris[wi];
      if (j >= 1 && coplanar(t, tris[seq[j - 1]])) continue;
      if (j + 1 <= k && coplanar(t, tris[seq[j]])) continue;
      const T x = plane_dist(t, Q[j]), y = plane_dist(t, Q[j + 1]);
      const T cross_plane = smooth(x, al, kind) * smooth(-y, al, kind) +
                            smooth(-x, al, kind) * smooth(y, al, kind);
      if (re(x) - re(y) == 0.0) continue;   // the leg's line never meets the plane
      const V3<T> hit = Q[j] + (x / (x - y)) * (Q[j + 1] - Q[j]);
      if (kind == SIGMOID) {
        // 1 - cross_plane inside = (1 - cross_plane) + cross_plane (1 - inside),
        // as in 2D: no cancellation where the triangle all but blocks the leg
        const T same_plane = smooth(x, al, kind) * smooth(y, al, kind) +
                             smooth(-x, al, kind) * smooth(-y, al, kind);
        visibility *= same_plane + cross_plane * outside(t, hit, al, kind);
      } else {
        visibility *= 1.0 - cross_plane * inside(t, hit, al, kind);
      }
    }
  }
  double gk = 1.0;
  for (int j = 0; j < k; ++j) gk *= P.gamma;
  return gk * validity * visibility / (L * L);
}

// an input value with its tangent (dropped for plain values)
template <class T>
T input(double v, double d);
template <>
double input<double>(double v, double) { return v; }
template <>
Dual input<Dual>(double v, double d) { return Dual(v, d); }

template <class T>
int power3_impl(const double* tris_xyz, const double* dtris, int W, const double* tx,
                const double* dtx, const double* rx, int R, int K, double alpha, int kind,
                double gamma, T* out) {
  std::vector<T> xyz(9 * W);
  for (int i = 0; i < 9 * W; ++i) xyz[i] = input<T>(tris_xyz[i], dtris ? dtris[i] : 0.0);
  std::vector<Tri<T>> tris;
  for (int i = 0; i < W; ++i) tris.push_back(make_tri<T>(&xyz[9 * i]));
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  const V3<T> t{input<T>(tx[0], dtx ? dtx[0] : 0.0), input<T>(tx[1], dtx ? dtx[1] : 0.0),
                input<T>(tx[2], dtx ? dtx[2] : 0.0)};
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    const V3<T> q{T(rx[3 * r]), T(rx[3 * r + 1]), T(rx[3 * r + 2])};
    T sum = T(0.0);
    for (const auto& seq : cands) sum += path_power3(tris, t, q, seq, prm);
    out[r] = sum;
  }
  return 0;
}

}  // namespace

extern "C" {

// Received power of a 3D triangle scene: tris [W][9] (A, B, C corners), tx [3], rx [R][3].
int drt_oracle_power3(const double* tris_xyz, int W, const double* tx, const double* rx, int R,
                      int K, double alpha, int kind, double gamma, int nthreads, double* Pw) {
  if (check_args(tris_xyz, W, tx, rx, R, K, alpha, kind)) return 1;
  set_threads(nthreads);
  return power3_impl<double>(tris_xyz, nullptr, W, tx, nullptr, rx, R, K, alpha, kind, gamma, Pw);
}

// Forward-mode derivative of the 3D power along (dtris [W][9], dtx [3]).
int drt_oracle_power3_jvp(const double* tris_xyz, int W, const double* tx, const double* rx,
                          int R, int K, double alpha, int kind, double gamma,
                          const double* dtris, const double* dtx, int nthreads, double* Pw,
                          double* dP) {
  if (check_args(tris_xyz, W, tx, rx, R, K, alpha, kind) || !dtris || !dtx) return 1;
  set_threads(nthreads);
  std::vector<Dual> out(R > 0 ? R : 1);
  const int rc = power3_impl<Dual>(tris_xyz, dtris, W, tx, dtx, rx, R, K, alpha, kind, gamma,
                                   out.data());
  for (int r = 0; r < R; ++r) {
    if (Pw) Pw[r] = out[r].v;
    dP[r] = out[r].d;
  }
  return rc;
}

// Number of path candidates for W walls and maximum order K.
long long drt_oracle_num_candidates(int W, int K) {
  long long n = 1, level = 1;
  for (int k = 1; k <= K; ++k) {
    level = (k == 1) ? W : level * (W - 1);
    n += level;
  }
  return n;
}

// Candidate table: seq_out [N][K] (unused slots -1), order_out [N].
int drt_oracle_candidates(int W, int K, int* seq_out, int* order_out) {
  auto c = candidates(W, K);
  for (size_t i = 0; i < c.size(); ++i) {
    order_out[i] = (int)c[i].size();
    for (int j = 0; j < K; ++j) seq_out[i * K + j] = j < (int)c[i].size() ? c[i][j] : -1;
  }
  return 0;
}

// Smoothing function and its derivative at x (dual number).
int drt_oracle_smooth(double x, double alpha, int kind, double* s, double* ds) {
  Dual r = smooth(Dual(x, 1.0), alpha, kind);
  *s = r.v;
  *ds = r.d;
  return 0;
}

// Received power P[r] for every receiver.
int drt_oracle_power(const double* walls_xy, int W, const double* tx, const double* rx, int R,
                     int K, double alpha, int kind, double gamma, int nthreads, double* P) {
  if (check_args(walls_xy, W, tx, rx, R, K, alpha, kind)) return 1;
  set_threads(nthreads);
  std::vector<double> xy(walls_xy, walls_xy + 4 * W);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<double> t{tx[0], tx[1]};
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    Vec<double> q{rx[2 * r], rx[2 * r + 1]};
    P[r] = received_power(walls, t, q, cands, prm);
  }
  return 0;
}

// Forward-mode derivative of every P[r] along the direction (dwalls [W][4], dtx [2]).
int drt_oracle_power_jvp(const double* walls_xy, int W, const double* tx, const double* rx,
                         int R, int K, double alpha, int kind, double gamma,
                         const double* dwalls, const double* dtx, int nthreads, double* P,
                         double* dP) {
  if (check_args(walls_xy, W, tx, rx, R, K, alpha, kind) || !dwalls || !dtx) return 1;
  set_threads(nthreads);
  std::vector<Dual> xy(4 * W);
  for (int i = 0; i < 4 * W; ++i) xy[i] = Dual(walls_xy[i], dwalls[i]);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<Dual> t{Dual(tx[0], dtx[0]), Dual(tx[1], dtx[1])};
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    Vec<Dual> q{Dual(rx[2 * r]), Dual(rx[2 * r + 1])};
    Dual v = received_power(walls, t, q, cands, prm);
    if (P) P[r] = v.v;
    dP[r] = v.d;
  }
  return 0;
}

// Complex-step derivative: Im P(x + i h dir) / h.
int drt_oracle_power_cstep(const double* walls_xy, int W, const double* tx, const double* rx,
                           int R, int K, double alpha, int kind, double gamma,
                           const double* dwalls, const double* dtx, double h, int nthreads,
                           double* dP) {
  if (check_args(walls_xy, W, tx, rx, R, K, alpha, kind) || !dwalls || !dtx) return 1;
  set_threads(nthreads);
  std::vector<Cplx> xy(4 * W);
  for (int i = 0; i < 4 * W; ++i) xy[i] = Cplx(walls_xy[i], h * dwalls[i]);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<Cplx> t{Cplx(tx[0], h * dtx[0]), Cplx(tx[1], h * dtx[1])};
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    Vec<Cplx> q{Cplx(rx[2 * r]), Cplx(rx[2 * r + 1])};
    Cplx v = received_power(walls, t, q, cands, prm);
    dP[r] = v.imag() / h;
  }
  return 0;
}

// Coherent field E[r] (re, im interleaved) summed over the candidate table in order;
// optionally mag[r] = sum of the path fields' magnitudes and lmax[r] = the longest
// path length with a non-zero field (the scales of FP32 rounding in E).
int drt_oracle_field(const double* walls_xy, int W, const double* tx, const double* rx, int R,
                     int K, double alpha, int kind, double gamma, double wavelength, double eps,
                     int nthreads, double* E, double* mag, double* lmax) {
  if (check_args(walls_xy, W, tx, rx, R, K, alpha, kind)) return 1;
  if (!(wavelength > 0.0) || !(eps == 0.0 || eps >= 1.0) || !(gamma >= 0.0)) return 1;
  set_threads(nthreads);
  std::vector<double> xy(walls_xy, walls_xy + 4 * W);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<double> t{tx[0], tx[1]};
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    Vec<double> q{rx[2 * r], rx[2 * r + 1]};
    double sre = 0.0, sim = 0.0;
    double m = 0.0, lm = 0.0;
    for (const auto& seq : cands) {
      double len = 0.0;
      const Vec<double> f = path_field(walls, t, q, seq, prm, wavelength, eps, &len);
      sre += f.x;
      sim += f.y;
      const double af = std::hypot(f.x, f.y);
      m += af;
      if (af > 0.0 && len > lm) lm = len;
    }
    E[2 * r] = sre;
    E[2 * r + 1] = sim;
    if (mag) mag[r] = m;
    if (lmax) lmax[r] = lm;
  }
  return 0;
}

// Forward-mode derivative of the coherent field along (dwalls [W][4], dtx [2]):
// E and dE (re, im interleaved) for every receiver.
int drt_oracle_field_jvp(const double* walls_xy, int W, const double* tx, const double* rx,
                         int R, int K, double alpha, int kind, double gamma, double wavelength,
                         double eps, const double* dwalls, const double* dtx, int nthreads,
                         double* E, double* dE) {
  if (check_args(walls_xy, W, tx, rx, R, K, alpha, kind) || !dwalls || !dtx) return 1;
  if (!(wavelength > 0.0) || !(eps == 0.0 || eps >= 1.0) || !(gamma >= 0.0)) return 1;
  set_threads(nthreads);
  std::vector<Dual> xy(4 * W);
  for (int i = 0; i < 4 * W; ++i) xy[i] = Dual(walls_xy[i], dwalls[i]);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<Dual> t{Dual(tx[0], dtx[0]), Dual(tx[1], dtx[1])};
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    Vec<Dual> q{Dual(rx[2 * r]), Dual(rx[2 * r + 1])};
    Dual sre(0.0), sim(0.0);
    for (const auto& seq : cands) {
      double len = 0.0;
      const Vec<Dual> f = path_field(walls, t, q, seq, prm, wavelength, eps, &len);
      sre = sre + f.x;
      sim = sim + f.y;
    }
    E[2 * r] = sre.v;
    E[2 * r + 1] = sim.v;
    dE[2 * r] = sre.d;
    dE[2 * r + 1] = sim.d;
  }
  return 0;
}

// Per-candidate detail for one receiver.  Arrays sized by the caller:
// degenerate [N], verts [N][K+2][2], validity [N], vis [N][K+1], length [N], power [N].
int drt_oracle_paths(const double* walls_xy, int W, const double* tx, const double* rx1, int K,
                     double alpha, int kind, double gamma, int* degenerate, double* verts,
                     double* validity, double* vis, double* length, double* power) {
  if (check_args(walls_xy, W, tx, rx1, 1, K, alpha, kind)) return 1;
  std::vector<double> xy(walls_xy, walls_xy + 4 * W);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<double> t{tx[0], tx[1]};
  Vec<double> q{rx1[0], rx1[1]};
  for (size_t i = 0; i < cands.size(); ++i) {
    PathRecord rec;
    for (int v = 0; v < 16; ++v) rec.verts[v] = NAN;
    for (int v = 0; v < 7; ++v) rec.vis[v] = NAN;
    path_power(walls, t, q, cands[i], prm, &rec);
    const int k = (int)cands[i].size();
    degenerate[i] = rec.degenerate;
    for (int v = 0; v < K + 2; ++v) {
      const bool used = v < k + 2;
      verts[(i * (K + 2) + v) * 2 + 0] = used ? rec.verts[2 * v] : NAN;
      verts[(i * (K + 2) + v) * 2 + 1] = used ? rec.verts[2 * v + 1] : NAN;
    }
    for (int j = 0; j < K + 1; ++j) vis[i * (K + 1) + j] = (j <= k && !rec.degenerate) ? rec.vis[j] : NAN;
    validity[i] = rec.validity;
    length[i] = rec.length;
    power[i] = rec.power;
  }
  return 0;
}


// Path-finder variant of drt_oracle_power (MPT points, convergence check): power [R].
int drt_oracle_power_finder(const double* walls_xy, int W, const double* tx, const double* rx,
                            int R, int K, double alpha, int kind, double gamma, int finder,
                            int n_iter, double eps, int nthreads, double* out) {
  if (check_args(walls_xy, W, tx, rx, R, K, alpha, kind) || n_iter < 0) return 1;
  if (finder != FINDER_MPT && finder != FINDER_FPT) return 1;
  std::vector<double> xy(walls_xy, walls_xy + 4 * W);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<double> t{tx[0], tx[1]};
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
  for (int r = 0; r < R; ++r) {
    Vec<double> q{rx[2 * r], rx[2 * r + 1]};
    double sum = 0.0;
    std::vector<double> tau;
    double C, kap;
    for (const auto& seq : cands)
      sum += finder_path_power(finder, walls, t, q, seq, prm, n_iter, eps, tau, &C, &kap);
    out[r] = sum;
  }
  return 0;
}

// Per path of one receiver: the finder's (0 MPT, 1 FPT) along-wall coordinates tau
// [n_cand][K] (NaN past the path's order and for a degenerate path), MPT cost C
// [n_cand], kappa [n_cand], power [n_cand], degenerate flag [n_cand].
int drt_oracle_finder_paths(const double* walls_xy, int W, const double* tx, const double* rx1,
                            int K, double alpha, int kind, double gamma, int finder, int n_iter,
                            double eps, double* tau_out, double* cost, double* kappa,
                            double* power, int* degenerate) {
  if (check_args(walls_xy, W, tx, rx1, 1, K, alpha, kind) || n_iter < 0) return 1;
  if (finder != FINDER_MPT && finder != FINDER_FPT) return 1;
  std::vector<double> xy(walls_xy, walls_xy + 4 * W);
  auto walls = make_walls(xy, W);
  auto cands = candidates(W, K);
  Params prm{K, alpha, kind, gamma};
  Vec<double> t{tx[0], tx[1]};
  Vec<double> q{rx1[0], rx1[1]};
  for (size_t i = 0; i < cands.size(); ++i) {
    std::vector<double> tau;
    const int k = (int)cands[i].size();
    power[i] = finder_path_power(finder, walls, t, q, cands[i], prm, n_iter, eps, tau, &cost[i],
                                 &kappa[i]);
    degenerate[i] = finder_points(finder, walls, t, q, cands[i], n_iter, tau) ? 0 : 1;
    for (int j = 0; j < K; ++j) tau_out[i * K + j] = (j < k && !degenerate[i]) ? tau[j] : NAN;
  }
  return 0;
}

}  // extern "C"
