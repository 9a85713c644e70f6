// Clebsch-Gordan layer of the SU(2) method: Wigner 6j (Eq. A3, triangle
// coefficient Eq. A4), 9j (Eq. A2) and the scalar factor C~ (Eq. a) of
// arXiv:2309.16724.  The 6j is evaluated exactly: every factorial is a
// vector of prime exponents, the terms of Racah's alternating sum share
// their common prime factors, and the remaining integers are summed in
// 128-bit arithmetic; only the final square root is rounded.
#include <cmath>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <unordered_map>

#include "su2_internal.h"

namespace su2 {
namespace {

constexpr int kPrimes[] = {2,  3,  5,  7,  11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53,
                           59, 61, 67, 71, 73, 79, 83, 89, 97, 101, 103, 107, 109, 113, 127, 131,
                           137, 139, 149, 151, 157, 163, 167, 173, 179, 181, 191, 193, 197, 199};
constexpr int kNP = sizeof(kPrimes) / sizeof(int);
constexpr int kMaxFact = 199;

struct PF {
  int e[kNP];
  PF() { std::memset(e, 0, sizeof(e)); }
};

// exponent of p in n! (Legendre)
PF fact_pf(int n) {
  if (n < 0 || n > kMaxFact) throw std::runtime_error("spin too large for the exact 6j");
  PF r;
  for (int i = 0; i < kNP; ++i) {
    int p = kPrimes[i], s = 0;
    for (long q = p; q <= n; q *= p) s += int(n / q);
    r.e[i] = s;
  }
  return r;
}

inline void add_to(PF& a, const PF& b, int sgn) {
  for (int i = 0; i < kNP; ++i) a.e[i] += sgn * b.e[i];
}

// value of a positive rational given by prime exponents, as a double
double pf_value(const PF& x) {
  unsigned __int128 num = 1, den = 1;
  bool exact = true;
  const unsigned __int128 lim = ~(unsigned __int128)0 / 256;
  for (int i = 0; i < kNP && exact; ++i) {
    int e = x.e[i];
    unsigned __int128& t = e > 0 ? num : den;
    for (int j = 0; j < (e > 0 ? e : -e); ++j) {
      if (t > lim) { exact = false; break; }
      t *= (unsigned)kPrimes[i];
    }
  }
  if (exact) return double(num) / double(den);
  double v = 1.0;  // rare: very large spins; product of exact prime powers
  for (int i = 0; i < kNP; ++i) v *= std::pow(double(kPrimes[i]), double(x.e[i]));
  return v;
}

double sixj_exact(int a, int b, int c, int d, int e, int f) {
  if (!(triangle(a, b, c) && triangle(c, d, e) && triangle(a, e, f) && triangle(b, d, f))) return 0.0;
  const int n2 = (a + b + c) / 2, n3 = (c + d + e) / 2, n4 = (a + e + f) / 2, n5 = (b + d + f) / 2;
  const int n6 = (a + b + d + e) / 2, n7 = (a + c + d + f) / 2, n8 = (b + c + e + f) / 2;
  int nmin = n2;
  if (n3 > nmin) nmin = n3;
  if (n4 > nmin) nmin = n4;
  if (n5 > nmin) nmin = n5;
  int nmax = n6;
  if (n7 < nmax) nmax = n7;
  if (n8 < nmax) nmax = n8;
  if (nmax < nmin) return 0.0;
  // squared prefactor: product of g~^2 over the four triads
  auto tri = [](int x, int y, int z, PF& acc) {
    add_to(acc, fact_pf((x + y - z) / 2), +1);
    add_to(acc, fact_pf((x - y + z) / 2), +1);
    add_to(acc, fact_pf((-x + y + z) / 2), +1);
    add_to(acc, fact_pf((x + y + z) / 2 + 1), -1);
  };
  PF pref;
  tri(a, b, c, pref);
  tri(c, d, e, pref);
  tri(a, e, f, pref);
  tri(b, d, f, pref);
  // terms (n+1)! / prod(...)!
  const int nt = nmax - nmin + 1;
  std::vector<PF> t(nt);
  for (int n = nmin; n <= nmax; ++n) {
    PF& x = t[n - nmin];
    add_to(x, fact_pf(n + 1), +1);
    add_to(x, fact_pf(n - n2), -1);
    add_to(x, fact_pf(n - n3), -1);
    add_to(x, fact_pf(n - n4), -1);
    add_to(x, fact_pf(n - n5), -1);
    add_to(x, fact_pf(n6 - n), -1);
    add_to(x, fact_pf(n7 - n), -1);
    add_to(x, fact_pf(n8 - n), -1);
  }
  PF common = t[0];
  for (int i = 1; i < nt; ++i)
    for (int j = 0; j < kNP; ++j)
      if (t[i].e[j] < common.e[j]) common.e[j] = t[i].e[j];
  __int128 sum = 0;
  const __int128 lim = (((__int128)1) << 120);
  for (int i = 0; i < nt; ++i) {
    __int128 u = 1;
    for (int j = 0; j < kNP; ++j)
      for (int r = 0; r < t[i].e[j] - common.e[j]; ++r) {
        u *= kPrimes[j];
        if (u > lim) throw std::runtime_error("exact 6j overflow");
      }
    sum += ((nmin + i) % 2 ? -u : u);
  }
  if (sum == 0) return 0.0;
  // value = sign(sum) * sqrt(pref * common^2) * |sum|
  PF sq = pref;
  add_to(sq, common, +2);
  const double mag = std::sqrt(pf_value(sq));
  const double s = double(sum < 0 ? -sum : sum);
  return (sum < 0 ? -1.0 : 1.0) * mag * s;
}

std::mutex g_mu;
std::unordered_map<uint64_t, double> g_sixj, g_ctilde;

uint64_t pack6(int a, int b, int c, int d, int e, int f) {
  return (uint64_t(a) << 50) | (uint64_t(b) << 40) | (uint64_t(c) << 30) | (uint64_t(d) << 20) |
         (uint64_t(e) << 10) | uint64_t(f);
}

}  // namespace

bool triangle(int a, int b, int c) {
  if (a < 0 || b < 0 || c < 0) return false;
  return std::abs(a - b) <= c && c <= a + b && ((a + b + c) % 2 == 0);
}

double sixj(int a, int b, int c, int d, int e, int f) {
  if (a > 1000 || b > 1000 || c > 1000 || d > 1000 || e > 1000 || f > 1000) return 0.0;
  const uint64_t key = pack6(a, b, c, d, e, f);
  {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_sixj.find(key);
    if (it != g_sixj.end()) return it->second;
  }
  const double v = sixj_exact(a, b, c, d, e, f);
  std::lock_guard<std::mutex> g(g_mu);
  g_sixj.emplace(key, v);
  return v;
}

double ninej(int j1, int j2, int j, int k1, int k2, int k, int j1p, int j2p, int jp) {
  if (!(triangle(j1, j2, j) && triangle(k1, k2, k) && triangle(j1p, j2p, jp) && triangle(j1, k1, j1p) &&
        triangle(j2, k2, j2p) && triangle(j, k, jp)))
    return 0.0;
  // x from max(|j1-j'|, |j2-k|, |k1-j2'|) to min(j1+j', j2+k, k1+j2'), step 1
  int xmin = std::abs(j1 - jp), t;
  if ((t = std::abs(j2 - k)) > xmin) xmin = t;
  if ((t = std::abs(k1 - j2p)) > xmin) xmin = t;
  int xmax = j1 + jp;
  if ((t = j2 + k) < xmax) xmax = t;
  if ((t = k1 + j2p) < xmax) xmax = t;
  double s = 0.0;
  for (int x = xmin; x <= xmax; x += 2) {
    const double sg = (x % 2) ? -1.0 : 1.0;  // (-1)^{2x}
    s += sg * (x + 1) *
         (sixj(j1, j2, j, k, jp, x) * sixj(k1, k2, k, j2, x, j2p) * sixj(j1p, j2p, jp, x, j1, k1));
  }
  return s;
}

double ctilde(int j1, int j2, int j, int k1, int k2, int k, int j1p, int j2p, int jp) {
  // key: nine twos values < 64 each
  if (j1 >= 64 || j2 >= 64 || j >= 64 || k1 >= 64 || k2 >= 64 || k >= 64 || j1p >= 64 || j2p >= 64 || jp >= 64) {
    const double w = ninej(j1, j2, j, k1, k2, k, j1p, j2p, jp);
    return w == 0.0 ? 0.0 : std::sqrt(double((j1p + 1) * (j2p + 1) * (j + 1) * (k + 1))) * w;
  }
  const uint64_t key = (uint64_t(j1) << 48) | (uint64_t(j2) << 42) | (uint64_t(j) << 36) | (uint64_t(k1) << 30) |
                       (uint64_t(k2) << 24) | (uint64_t(k) << 18) | (uint64_t(j1p) << 12) | (uint64_t(j2p) << 6) |
                       uint64_t(jp);
  {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_ctilde.find(key);
    if (it != g_ctilde.end()) return it->second;
  }
  const double w = ninej(j1, j2, j, k1, k2, k, j1p, j2p, jp);
  // Eq. a: sqrt((2j1'+1)(2j2'+1)(2j+1)(2k+1)) W9j; primed = output side
  const double v = (w == 0.0) ? 0.0 : std::sqrt(double((j1p + 1) * (j2p + 1) * (j + 1) * (k + 1))) * w;
  std::lock_guard<std::mutex> g(g_mu);
  g_ctilde.emplace(key, v);
  return v;
}

// ------------------------------------------------------------------ Clebsch-Gordan
static double fct(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// <j1 m1; j2 m2 | J M> by Racah's closed form (twos arguments)
double cg_coef(int j1, int m1, int j2, int m2, int J, int M) {
  if (m1 + m2 != M || !triangle(j1, j2, J)) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(M) > J) return 0.0;
  if ((j1 + m1) % 2 || (j2 + m2) % 2 || (J + M) % 2) return 0.0;
  const int a = (j1 + j2 - J) / 2, b = (j1 - j2 + J) / 2, c = (-j1 + j2 + J) / 2, d = (j1 + j2 + J) / 2 + 1;
  double pre = (J + 1) * fct(a) * fct(b) * fct(c) / fct(d);
  pre *= fct((J + M) / 2) * fct((J - M) / 2) * fct((j1 - m1) / 2) * fct((j1 + m1) / 2) * fct((j2 - m2) / 2) *
         fct((j2 + m2) / 2);
  double sum = 0.0;
  for (int k = 0; k <= a; ++k) {
    const int x1 = (j1 - m1) / 2 - k, x2 = (j2 + m2) / 2 - k, x3 = (J - j2 + m1) / 2 + k, x4 = (J - j1 - m2) / 2 + k;
    if (x1 < 0 || x2 < 0 || x3 < 0 || x4 < 0) continue;
    const double t = 1.0 / (fct(k) * fct(a - k) * fct(x1) * fct(x2) * fct(x3) * fct(x4));
    sum += (k % 2) ? -t : t;
  }
  return std::sqrt(pre) * sum;
}


}  // namespace su2
