"""The oracle's pins must catch plausible mistakes.

Each mutant is a copy of the oracle source with one planted mistake (a flipped
sign, a dropped term, a wrong index, a transposed operand).  It is compiled on
the CPU into a temporary directory and the oracle pin tests run against it in
a subprocess; every mutant must make at least one pin fail.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "drt_oracle.cpp")
PIN_FILES = ["tests/test_oracle_smoothing.py", "tests/test_oracle_candidates.py",
             "tests/test_oracle_geometry.py", "tests/test_oracle_bruteforce.py",
             "tests/test_oracle_gradients.py", "tests/test_oracle_field.py",
             "tests/test_oracle_3d.py", "tests/test_oracle_mpt_finder.py",
             "tests/test_oracle_fpt_finder.py", "tests/test_oracle_deep_shadow.py"]

MUTANTS = {
    "mirror sign": ("return Vec<T>{p.x - 2.0 * d * w.n.x", "return Vec<T>{p.x + 2.0 * d * w.n.x"),
    "normal not perpendicular": ("w.n = Vec<T>{-w.u.y, w.u.x};", "w.n = Vec<T>{w.u.y, w.u.x};"),
    "backtrace ratio": ("T t = b / (b - a);", "T t = a / (b - a);"),
    "exclusion drops one wall": ("if (wi == skip_a || wi == skip_b) continue;",
                                 "if (wi == skip_a) continue;"),
    "no exclusion": ("if (wi == skip_a || wi == skip_b) continue;", ""),
    "exclusion wrong index": ("const int skip_b = (j + 1 <= k) ? seq[j] : -1;",
                              "const int skip_b = (j + 1 <= k) ? seq[k - 1] : -1;"),
    "crossing test sign": ("T cross1 = smooth(x1, a, kind) * smooth(T(-y1), a, kind) +",
                           "T cross1 = smooth(x1, a, kind) * smooth(y1, a, kind) +"),
    "tip test uses A twice": ("T y2 = dot(leg_normal[j], sub(w.b, Q[j]));",
                              "T y2 = dot(leg_normal[j], sub(w.a, Q[j]));"),
    "leg tangent for normal": ("leg_normal[j] = Vec<T>{-d.y / l, d.x / l};",
                               "leg_normal[j] = Vec<T>{d.x / l, d.y / l};"),
    "same-side term": ("smooth(T(-p), a, kind) * smooth(T(-q), a, kind);",
                       "smooth(T(-p), a, kind) * smooth(q, a, kind);"),
    "on-segment far end": ("smooth(w.len - tj, a, kind)", "smooth(tj - w.len, a, kind)"),
    "validity drops side test": ("validity = validity * on_seg * same_side;",
                                 "validity = validity * on_seg;"),
    "blocked product to sum": ("vis = vis * (1.0 - cross1 * cross2);",
                               "vis = vis * (1.0 - cross1);"),
    "inverse length not squared": ("T power = gk * validity * visibility / (L * L);",
                                   "T power = gk * validity * visibility / L;"),
    "no reflection coefficient": ("for (int j = 0; j < k; ++j) gk *= P.gamma;",
                                  "for (int j = 0; j < k; ++j) gk *= 1.0;"),
    "hard sigmoid slope": ("return y / 6.0;", "return y / 3.0;"),
    "sigmoid sign": ("return 1.0 / (1.0 + exp(-z));", "return 1.0 / (1.0 + exp(z));"),
    "step tie": ("return T(re(x) > 0.0 ? 1.0 : 0.0);", "return T(re(x) >= 0.0 ? 1.0 : 0.0);"),
    "repeat allowed": ("if (!s.empty() && s.back() == w) continue;", ""),
    "dual quotient rule": ("(a.d * b.v - a.v * b.d) / (b.v * b.v)",
                           "(a.d * b.v + a.v * b.d) / (b.v * b.v)"),
    "dual exp": ("return Dual(e, a.d * e);", "return Dual(e, a.d);"),
    "field phase sign": ("return Vec<T>{amp * cos(phase), -(amp * sin(phase))};",
                         "return Vec<T>{amp * cos(phase), amp * sin(phase)};"),
    "field wavelength factor": ("const T phase = (2.0 * M_PI / wavelength) * t.L;",
                                "const T phase = (M_PI / wavelength) * t.L;"),
    "field spreading squared": ("const T amp = coef * t.validity * t.visibility / t.L;",
                                "const T amp = coef * t.validity * t.visibility / (t.L * t.L);"),
    "fresnel numerator sign": ("return (c - r) / (c + r);", "return (r - c) / (c + r);"),
    "fresnel sine for cosine": ("const T r = sqrt(eps - (1.0 - c * c));",
                                "const T r = sqrt(eps - c * c);"),
    "constant coefficient sign": ("T(-std::sqrt(P.gamma))", "T(std::sqrt(P.gamma))"),
    "dual cosine derivative": ("return Dual(std::cos(a.v), -a.d * std::sin(a.v));",
                               "return Dual(std::cos(a.v), a.d * std::sin(a.v));"),
    "dual sine derivative": ("return Dual(std::sin(a.v), a.d * std::cos(a.v));",
                             "return Dual(std::sin(a.v), a.d * std::sin(a.v));"),
    "3d mirror sign": ("img[j] = img[j - 1] - (2.0 * plane_dist(t, img[j - 1])) * t.n;",
                       "img[j] = img[j - 1] + (2.0 * plane_dist(t, img[j - 1])) * t.n;"),
    "3d inside tests two edges": ("for (int k = 0; k < 3; ++k) r *= smooth(edge_dist(t, k, p), alpha, kind);",
                                  "for (int k = 0; k < 2; ++k) r *= smooth(edge_dist(t, k, p), alpha, kind);"),
    "3d edge normals outward": ("t.m[k] = (1.0 / norm(e)) * cross(t.n, e);",
                                "t.m[k] = (1.0 / norm(e)) * cross(e, t.n);"),
    "3d crossing point": ("const V3<T> hit = Q[j] + (x / (x - y)) * (Q[j + 1] - Q[j]);",
                          "const V3<T> hit = Q[j] + (y / (x - y)) * (Q[j + 1] - Q[j]);"),
    "3d crossing test sign": ("const T cross_plane = smooth(x, al, kind) * smooth(-y, al, kind) +",
                              "const T cross_plane = smooth(x, al, kind) * smooth(y, al, kind) +"),
    "3d same-side term": ("smooth(-p, al, kind) * smooth(-q, al, kind);",
                          "smooth(-p, al, kind) * smooth(q, al, kind);"),
    "3d coplanar pair kept": ("if (coplanar(tris[seq[j - 1]], tris[seq[j]])) return T(0.0);",
                              "if (false) return T(0.0);"),
    "3d coplanar triangles tested": ("if (j >= 1 && coplanar(t, tris[seq[j - 1]])) continue;",
                                     "if (j >= 1 && &t == &tris[seq[j - 1]]) continue;"),
    "mpt residual mirror sign": ("hout.x - (hin.x - 2.0 * in * w.n.x)",
                                 "hout.x - (hin.x + 2.0 * in * w.n.x)"),
    "mpt jacobian drops the incoming leg": (
        "J[(j - 1) * k + (j - 1)] = Vec<double>{-a.x - c.x, -a.y - c.y};",
        "J[(j - 1) * k + (j - 1)] = Vec<double>{-a.x, -a.y};"),
    "mpt check compares the wrong way": ("*kappa = smooth(eps - *cost, P.alpha, P.kind);",
                                          "*kappa = smooth(*cost - eps, P.alpha, P.kind);"),
    "mpt on-segment far end": ("smooth(w.len - tau[j - 1], P.alpha, P.kind);",
                               "smooth(tau[j - 1] - w.len, P.alpha, P.kind);"),
    "mpt line search takes increases": (
        "if (mpt_cost(walls, seq, ft) <= C0 + 1e-4 * t * slope + tol) {",
        "if (mpt_cost(walls, seq, ft) >= C0 + 1e-4 * t * slope + tol) {"),
    "fpt gradient sign": ("b[j - 1] = -(dot(u, f.h[j - 1]) - dot(u, f.h[j]));",
                          "b[j - 1] = (dot(u, f.h[j - 1]) - dot(u, f.h[j]));"),
    "fpt hessian coupling sign": ("const double c = -pquad(f, j, u, walls[seq[j]].u);",
                                  "const double c = pquad(f, j, u, walls[seq[j]].u);"),
    "fpt hessian drops the outgoing leg": ("pquad(f, j - 1, u, u) + pquad(f, j, u, u)",
                                           "pquad(f, j - 1, u, u)"),
    "fpt line search takes increases": ("if (length(ft) <= L0 + 1e-4 * t * slope + tol)",
                                        "if (length(ft) >= L0 + 1e-4 * t * slope + tol)"),
    "mpt keeps paths with a vanishing leg": ("if (l < MPT_MIN_LEG) return false;", ""),
    "sigmoid obstruction formed with cancellation": ("vis = vis * (same1 + cross1 * same2);",
                                                     "vis = vis * (1.0 - cross1 * cross2);"),
    "sigmoid same-side complement sign": ("T same2 = smooth(x2, a, kind) * smooth(y2, a, kind) +",
                                          "T same2 = smooth(x2, a, kind) * smooth(T(-y2), a, kind) +"),
    "3d sigmoid obstruction formed with cancellation": (
        "visibility *= same_plane + cross_plane * outside(t, hit, al, kind);",
        "visibility *= 1.0 - cross_plane * inside(t, hit, al, kind);"),
    "3d outside drops a term": ("smooth(d1, alpha, kind) * smooth(T(-d2), alpha, kind));",
                                "T(0.0));"),
    "along from B": ("T along(const Wall<T>& w, const Vec<T>& p) { return dot(w.u, sub(p, w.a)); }",
                     "T along(const Wall<T>& w, const Vec<T>& p) { return dot(w.u, sub(p, w.b)); }"),
}


def _build(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutant {name!r} no longer matches the oracle source"
    mutated = src.replace(old, new, 1)
    path = os.path.join(tmp, name.replace(" ", "_"))
    with open(path + ".cpp", "w") as f:
        f.write(mutated)
    subprocess.run(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o",
                    path + ".so", path + ".cpp"], check=True)
    env = dict(os.environ, DRT_ORACLE_LIB=path + ".so", OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *PIN_FILES], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode


def test_every_mutant_is_caught():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=max(2, (os.cpu_count() or 2))) as ex:
            futs = {name: ex.submit(_build, name, old, new, tmp)
                    for name, (old, new) in MUTANTS.items()}
            survivors = [name for name, f in futs.items() if f.result() == 0]
    assert not survivors, f"mutants not caught by any pin: {survivors}"
