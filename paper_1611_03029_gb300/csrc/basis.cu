// Host-side 1D reference-element tables on [0, 1] (Sec. 2.1, Sec. 3),
// computed once in long double and rounded to float64 / float32.
#include <cmath>
#include <mutex>

#include "mfp_internal.h"

namespace mfp {
namespace {

using ld = long double;

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, ld x, ld& P, ld& dP) {
  ld p0 = 1, p1 = x;
  if (n == 0) {
    P = 1;
    dP = 0;
    return;
  }
  for (int m = 1; m < n; ++m) {
    ld p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  // n (x P_n - P_{n-1}) / (x^2 - 1); only used away from +-1
  dP = n * (x * p1 - p0) / (x * x - 1);
}

// Gauss-Legendre points / weights on [-1, 1]: roots of P_n by Newton.
void gauss(int n, ld* x, ld* w) {
  const ld pi = 3.14159265358979323846264338327950288L;
  for (int i = 0; i < n; ++i) {
    ld t = -std::cos(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(n, t, P, dP);
      ld dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-19L) break;
    }
    ld P, dP;
    legendre(n, t, P, dP);
    x[i] = t;
    w[i] = 2 / ((1 - t * t) * dP * dP);
  }
}

// Gauss-Lobatto points on [-1, 1]: +-1 and the roots of P_k', by Newton with
// P_k'' from Legendre's equation (1-x^2) P'' = 2 x P' - k(k+1) P.
void lobatto(int k, ld* x) {
  const ld pi = 3.14159265358979323846264338327950288L;
  x[0] = -1;
  x[k] = 1;
  for (int i = 1; i < k; ++i) {
    ld t = -std::cos(pi * i / k);
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(k, t, P, dP);
      ld d2P = (2 * t * dP - k * (k + 1) * P) / (1 - t * t);
      ld dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-19L) break;
    }
    x[i] = t;
  }
}

ld lagrange(const ld* nodes, int n, int j, ld x) {
  ld v = 1;
  for (int m = 0; m < n; ++m)
    if (m != j) v *= (x - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

ld lagrange_deriv(const ld* nodes, int n, int j, ld x) {
  ld s = 0;
  for (int m = 0; m < n; ++m) {
    if (m == j) continue;
    ld t = 1 / (nodes[j] - nodes[m]);
    for (int l = 0; l < n; ++l)
      if (l != j && l != m) t *= (x - nodes[l]) / (nodes[j] - nodes[l]);
    s += t;
  }
  return s;
}

template <typename T>
void fill(DevTab<T>& t, int k) {
  const int p = k + 1;
  ld xl[kMaxP], xg[kMaxP], wg[kMaxP];
  lobatto(k, xl);
  gauss(p, xg, wg);
  // map to [0, 1]
  for (int i = 0; i < p; ++i) {
    xl[i] = (xl[i] + 1) / 2;
    xg[i] = (xg[i] + 1) / 2;
    wg[i] = wg[i] / 2;
  }
  for (int i = 0; i < kMaxP * kMaxP; ++i)
    t.S[i] = t.D[i] = t.Dphi[i] = t.E0[i] = t.E1[i] = 0;
  for (int i = 0; i < kMaxP; ++i) t.dphi0[i] = t.dphi1[i] = t.w[i] = 0;
  for (int q = 0; q < p; ++q) {
    t.w[q] = (T)wg[q];
    t.g[q] = (T)xg[q];
    t.x[q] = (T)xl[q];
    for (int j = 0; j < p; ++j) {
      t.S[q * p + j] = (T)lagrange(xl, p, j, xg[q]);
      t.Dphi[q * p + j] = (T)lagrange_deriv(xl, p, j, xg[q]);
      t.D[q * p + j] = (T)lagrange_deriv(xg, p, j, xg[q]);
      t.E0[q * p + j] = (T)lagrange(xl, p, j, xl[q] / 2);
      t.E1[q * p + j] = (T)lagrange(xl, p, j, (1 + xl[q]) / 2);
    }
  }
  for (int j = 0; j < p; ++j) {
    t.dphi0[j] = (T)lagrange_deriv(xl, p, j, 0.0L);
    t.dphi1[j] = (T)lagrange_deriv(xl, p, j, 1.0L);
  }
  for (int i = 0; i < kMaxP; ++i) t.gv0[i] = t.gv1[i] = t.gd0[i] = t.gd1[i] = 0;
  for (int q = 0; q < p; ++q) {
    t.gv0[q] = (T)lagrange(xg, p, q, 0.0L);
    t.gv1[q] = (T)lagrange(xg, p, q, 1.0L);
    t.gd0[q] = (T)lagrange_deriv(xg, p, q, 0.0L);
    t.gd1[q] = (T)lagrange_deriv(xg, p, q, 1.0L);
  }
}

}  // namespace

const HostTables& host_tables() {
  static HostTables tabs;
  static std::once_flag once;
  std::call_once(once, [] {
    for (int k = 1; k <= 8; ++k) {
      fill(tabs.d[k - 1], k);
      fill(tabs.f[k - 1], k);
      const DevTab<double>& d = tabs.d[k - 1];
      DevTabDF& t = tabs.df[k - 1];
      auto split = [](double v, float& h, float& l) {
        h = (float)v;
        l = (float)(v - (double)h);
      };
      for (int i = 0; i < kMaxP * kMaxP; ++i) {
        split(d.S[i], t.Sh[i], t.Sl[i]);
        split(d.D[i], t.Dh[i], t.Dl[i]);
      }
      for (int i = 0; i < kMaxP; ++i) {
        split(d.dphi0[i], t.d0h[i], t.d0l[i]);
        split(d.dphi1[i], t.d1h[i], t.d1l[i]);
        split(d.w[i], t.wh[i], t.wl[i]);
      }
      // even-odd split of S, D and their transposes
      {
        const int p = k + 1, h = p / 2, mc = h + p % 2;
        DevTabEO& e = tabs.eo[k - 1];
        for (int w = 0; w < 4; ++w) {
          const double* M = (w / 2) ? d.D : d.S;
          const bool tr = w % 2;
          auto m = [&](int q, int j) {
            return tr ? M[j * p + q] : M[q * p + j];
          };
          for (int i = 0; i < kMaxH * kMaxH; ++i)
            e.ah[w][i] = e.al[w][i] = e.bh[w][i] = e.bl[w][i] = 0.f;
          for (int q = 0; q < mc; ++q) {
            for (int j = 0; j < h; ++j) {
              split(0.5 * (m(q, j) + m(q, p - 1 - j)), e.ah[w][q * kMaxH + j],
                    e.al[w][q * kMaxH + j]);
              split(0.5 * (m(q, j) - m(q, p - 1 - j)), e.bh[w][q * kMaxH + j],
                    e.bl[w][q * kMaxH + j]);
            }
            if (p % 2)
              split(m(q, h), e.ah[w][q * kMaxH + h], e.al[w][q * kMaxH + h]);
          }
        }
      }
      // Gauss-point Lagrange basis at the ends of [0, 1]
      for (int q = 0; q < kMaxP; ++q) {
        split(d.gv0[q], t.gv0h[q], t.gv0l[q]);
        split(d.gv1[q], t.gv1h[q], t.gv1l[q]);
        split(d.gd0[q], t.gd0h[q], t.gd0l[q]);
        split(d.gd1[q], t.gd1h[q], t.gd1l[q]);
      }
    }
  });
  return tabs;
}

}  // namespace mfp
