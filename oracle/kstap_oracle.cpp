// Kron-STAP FP64 oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct CPU restatement of what Greenewald, Zelnio
// and Hero, "Kronecker STAP and SAR GMTI" define, used to check the CUDA path.
// Only the tests, the smoke check and the benchmark's CPU-baseline leg may call
// it; the product path never links or loads it.  It shares no code, header or
// helper with the CUDA library.
//
// Steps (paper notation; 0-based indices in code, 1-based in Alg. 1):
//   O1  snapshots: X[i][j] = Y_i(r + Rr, c + Ra + j), x = vec(X^T)   (Sec. 2)
//       training set = cells (r+dr, c+dc) of the (2Rr+1)x(2Ra+1) box minus
//       the (2Gr+1)x(2Ga+1) guard box (n cells).
//   O2  S = (1/n) sum_m x_m x_m^H                       (Eq. SCM; the x x^T
//       printed in Alg. 2 is read as x x^H)
//   O3  R = Rearrange(S) by Alg. 1, run literally with 1-based indices.
//   O4  a_0 = R 1_{q^2} / q^2                            (Sec. 4 init; the
//       1_{q x 1} printed there is read as 1_{q^2 x 1})
//   O5  Alg. 2 loop: b = R^T conj(a)/|a|^2 ; a~ = R conj(b)/|b|^2 ;
//       a = vec(EIG_{r_a}(vec^-1 a~)) ; eta = |R - a b^T|_F / |R|_F, explicit.
//       Stop when |eta_k - eta_{k-1}| <= eps (eta_0 = +inf) or k = max_iter.
//   O6  A^ = vec^-1(a), B^ = EIG_{r_b}(vec^-1 b) with b the last computed b.
//       U_A, U_B = leading eigenvectors from this file's cyclic Jacobi.
//   O7  P = (I - U_A U_A^H) (x) (I - U_B U_B^H) formed densely (Eq. KronSTAP),
//       T_v = |d_v^H P x|^2 / (d_v^H P d_v), d_v = a_v (x) b_v / sqrt(pq);
//       T_v = 0 when d_v^H P d_v < 1e-12 |d_v|^2.
//       Tmax = max_v T_v, vidx = lowest maximising v, map = Tmax > tau.
//       filter = 1 selects the classical projector of Sec. 5 instead:
//       P = I - (U_A (x) U_B)(U_A (x) U_B)^H, formed densely the same way.
// EIG_r keeps the r algebraically largest eigenpairs (Sec. 4 definition;
// for the PSD matrices that occur they are also the largest in magnitude).
// Hermitian inputs to EIG are first symmetrised, herm(M) = (M + M^H)/2.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cd;

namespace {

// ---------------------------------------------------------------- Jacobi ----
// Cyclic complex Jacobi for an n x n Hermitian matrix M (row-major, destroyed).
// On return w[0..n-1] holds the eigenvalues in decreasing order and the
// columns of U (row-major n x n) the matching orthonormal eigenvectors.
// Each rotation removes the phase of M_pq with a diagonal unitary and then
// applies the real symmetric Jacobi rotation (t = tan theta,
// cot 2 theta = (M_qq - M_pp) / (2 |M_pq|)).
void jacobi_herm(std::vector<cd>& M, int n, std::vector<double>& w, std::vector<cd>& U) {
  U.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) U[(size_t)i * n + i] = 1.0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      cd h = 0.5 * (M[(size_t)i * n + j] + std::conj(M[(size_t)j * n + i]));
      M[(size_t)i * n + j] = h;
      M[(size_t)j * n + i] = std::conj(h);
    }
  for (int i = 0; i < n; ++i) M[(size_t)i * n + i] = M[(size_t)i * n + i].real();
  double fro = 0;
  for (auto& v : M) fro += std::norm(v);
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off += std::norm(M[(size_t)i * n + j]);
    if (fro == 0.0 || std::sqrt(off) <= 1e-15 * fro) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        cd b = M[(size_t)p * n + q];
        double ab = std::abs(b);
        if (ab == 0.0) continue;
        double a = M[(size_t)p * n + p].real();
        double d = M[(size_t)q * n + q].real();
        cd ph = b / ab;  // e^{i phi}
        double tau = (d - a) / (2.0 * ab);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t);
        double s = t * c;
        // G = diag(1, conj(ph)) [[c, s], [-s, c]]
        cd g_pp = c, g_pq = s, g_qp = -s * std::conj(ph), g_qq = c * std::conj(ph);
        for (int k = 0; k < n; ++k) {  // M <- M G
          cd mp = M[(size_t)k * n + p], mq = M[(size_t)k * n + q];
          M[(size_t)k * n + p] = mp * g_pp + mq * g_qp;
          M[(size_t)k * n + q] = mp * g_pq + mq * g_qq;
        }
        for (int k = 0; k < n; ++k) {  // M <- G^H M
          cd mp = M[(size_t)p * n + k], mq = M[(size_t)q * n + k];
          M[(size_t)p * n + k] = std::conj(g_pp) * mp + std::conj(g_qp) * mq;
          M[(size_t)q * n + k] = std::conj(g_pq) * mp + std::conj(g_qq) * mq;
        }
        M[(size_t)p * n + q] = 0.0;
        M[(size_t)q * n + p] = 0.0;
        M[(size_t)p * n + p] = M[(size_t)p * n + p].real();
        M[(size_t)q * n + q] = M[(size_t)q * n + q].real();
        for (int k = 0; k < n; ++k) {  // U <- U G
          cd up = U[(size_t)k * n + p], uq = U[(size_t)k * n + q];
          U[(size_t)k * n + p] = up * g_pp + uq * g_qp;
          U[(size_t)k * n + q] = up * g_pq + uq * g_qq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::vector<double> d(n);
  for (int i = 0; i < n; ++i) d[i] = M[(size_t)i * n + i].real();
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return d[x] > d[y]; });
  w.resize(n);
  std::vector<cd> Us((size_t)n * n);
  for (int k = 0; k < n; ++k) {
    w[k] = d[order[k]];
    for (int i = 0; i < n; ++i) Us[(size_t)i * n + k] = U[(size_t)i * n + order[k]];
  }
  U.swap(Us);
}

// EIG_r(M) = sum_{i<r} w_i u_i u_i^H (row-major n x n), plus the eigenpairs.
void eig_trunc(const std::vector<cd>& Min, int n, int r, std::vector<cd>& out,
               std::vector<double>& w, std::vector<cd>& U) {
  std::vector<cd> M(Min);
  jacobi_herm(M, n, w, U);
  out.assign((size_t)n * n, cd(0, 0));
  for (int k = 0; k < r; ++k)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        out[(size_t)i * n + j] += w[k] * U[(size_t)i * n + k] * std::conj(U[(size_t)j * n + k]);
}

// ------------------------------------------------------------- Alg. 1 ------
// R (p^2 x q^2, row-major) from S (pq x pq, row-major) by the paper's index
// formula, with 1-based P in 1..q^2 (columns) and J in 1..p^2 (rows).
void rearrange_alg1(const std::vector<cd>& S, int p, int q, std::vector<cd>& R) {
  const long pq = (long)p * q;
  // s = vec(S), column-major: s_M (1-based) = S(row (M-1) mod pq, col (M-1) div pq)
  auto s_at = [&](long M) -> cd {
    long m0 = M - 1;
    return S[(size_t)(m0 % pq) * pq + (m0 / pq)];
  };
  R.assign((size_t)p * p * q * q, cd(0, 0));
  for (long i = 1; i <= (long)q * q; ++i)
    for (long j = 1; j <= (long)p * p; ++j) {
      const long P = i, J = j;
      const long L = P - q * ((P - 1) / q) + q * (J - p * ((J - 1) / p) - 1);
      const long N = (P + q - 1) / q + q * ((J + p - 1) / p - 1);  // ceil(P/q) + q(ceil(J/p)-1)
      const long M = L + (N - 1) * pq;
      R[(size_t)(J - 1) * q * q + (P - 1)] = s_at(M);
    }
}

double fro2(const std::vector<cd>& v) {
  double s = 0;
  for (auto& x : v) s += std::norm(x);
  return s;
}

struct LRKronResult {
  std::vector<cd> A, B;          // A^ (p x p), B^ (q x q), row-major, tr A^ = p
  std::vector<cd> UA, UB;        // p x r_a, q x r_b (row-major)
  std::vector<double> lamA, lamB;
  std::vector<double> wB_all;    // all eigenvalues of herm(vec^-1 b), decreasing
  int iters = 0;
  double eta = 0;
  std::vector<double> eta_hist;
};

// Alg. 2 on a given S (pq x pq row-major).
void lrkron(const std::vector<cd>& S, int p, int q, int r_a, int r_b, double eps, int max_iter,
            LRKronResult& res) {
  const int p2 = p * p, q2 = q * q;
  std::vector<cd> R;
  rearrange_alg1(S, p, q, R);
  const double Rn = std::sqrt(fro2(R));
  std::vector<cd> a(p2, cd(0, 0));  // a_0 = R 1 / q^2
  for (int J = 0; J < p2; ++J) {
    cd s = 0;
    for (int P = 0; P < q2; ++P) s += R[(size_t)J * q2 + P];
    a[J] = s / double(q2);
  }
  std::vector<cd> b(q2), at(p2), Am((size_t)p2), Atr;
  std::vector<double> w;
  std::vector<cd> U;
  double eta_prev = std::numeric_limits<double>::infinity();
  int k = 0;
  res.eta_hist.clear();
  while (true) {
    const double an = fro2(a);
    for (int P = 0; P < q2; ++P) {  // b_k = R^T conj(a_k) / |a_k|^2
      cd s = 0;
      for (int J = 0; J < p2; ++J) s += R[(size_t)J * q2 + P] * std::conj(a[J]);
      b[P] = s / an;
    }
    const double bn = fro2(b);
    for (int J = 0; J < p2; ++J) {  // a~ = R conj(b_k) / |b_k|^2
      cd s = 0;
      for (int P = 0; P < q2; ++P) s += R[(size_t)J * q2 + P] * std::conj(b[P]);
      at[J] = s / bn;
    }
    for (int i = 0; i < p; ++i)  // vec^-1 (column-major): A(i, j) = a[i + p j]
      for (int j = 0; j < p; ++j) Am[(size_t)i * p + j] = at[i + p * j];
    eig_trunc(Am, p, r_a, Atr, w, U);  // a_{k+1} = vec(EIG_{r_a}(.))
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) a[i + p * j] = Atr[(size_t)i * p + j];
    double e2 = 0;  // eta_{k+1} = |R - a_{k+1} b_k^T|_F / |R|_F
    for (int J = 0; J < p2; ++J)
      for (int P = 0; P < q2; ++P) e2 += std::norm(R[(size_t)J * q2 + P] - a[J] * b[P]);
    const double eta = (Rn > 0) ? std::sqrt(e2) / Rn : 0.0;
    res.eta_hist.push_back(eta);
    ++k;
    const bool done = (std::fabs(eta - eta_prev) <= eps) || (k >= max_iter);
    eta_prev = eta;
    if (done) break;
  }
  res.iters = k;
  res.eta = eta_prev;
  std::vector<cd> Ah((size_t)p * p), Bm((size_t)q * q), Bh;
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) Ah[(size_t)i * p + j] = a[i + p * j];
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) Bm[(size_t)i * q + j] = b[i + q * j];
  std::vector<double> wA, wB;
  std::vector<cd> UAf, UBf;
  {
    std::vector<cd> tmp(Ah);
    jacobi_herm(tmp, p, wA, UAf);
  }
  eig_trunc(Bm, q, r_b, Bh, wB, UBf);  // B^ = EIG_{r_b}(vec^-1 b)
  double trA = 0;  // trace normalisation tr A^ = p (the scale is not identifiable)
  for (int i = 0; i < p; ++i) trA += Ah[(size_t)i * p + i].real();
  const double sc = (trA != 0) ? double(p) / trA : 1.0;
  res.A.resize((size_t)p * p);
  res.B.resize((size_t)q * q);
  for (size_t i = 0; i < Ah.size(); ++i) res.A[i] = Ah[i] * sc;
  for (size_t i = 0; i < Bh.size(); ++i) res.B[i] = Bh[i] / sc;
  res.UA.assign((size_t)p * r_a, cd(0, 0));
  res.UB.assign((size_t)q * r_b, cd(0, 0));
  for (int i = 0; i < p; ++i)
    for (int m = 0; m < r_a; ++m) res.UA[(size_t)i * r_a + m] = UAf[(size_t)i * p + m];
  for (int i = 0; i < q; ++i)
    for (int m = 0; m < r_b; ++m) res.UB[(size_t)i * r_b + m] = UBf[(size_t)i * q + m];
  res.lamA.resize(r_a);
  res.lamB.resize(r_b);
  for (int m = 0; m < r_a; ++m) res.lamA[m] = wA[m] * sc;
  for (int m = 0; m < r_b; ++m) res.lamB[m] = wB[m] / sc;
  res.wB_all.resize(q);
  for (int m = 0; m < q; ++m) res.wB_all[m] = wB[m] / sc;
}

// Dense Kron-STAP statistic (O7) for snapshot x (pq) and projector factors;
// filter 0 = F_A (x) F_B (Eq. KronSTAP), 1 = the classical I - W W^H with
// W = U_A (x) U_B (Sec. 5).
void kstap_stat(const std::vector<cd>& x, const std::vector<cd>& UA, const std::vector<cd>& UB,
                int p, int q, int r_a, int r_b, const std::vector<cd>& bank_a,
                const std::vector<cd>& bank_b, int V, double* T, double* cond, int filter) {
  const int n = p * q;
  std::vector<cd> FA((size_t)p * p), FB((size_t)q * q), P((size_t)n * n);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      cd s = (i == j) ? 1.0 : 0.0;
      for (int m = 0; m < r_a; ++m) s -= UA[(size_t)i * r_a + m] * std::conj(UA[(size_t)j * r_a + m]);
      FA[(size_t)i * p + j] = s;
    }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      cd s = (i == j) ? 1.0 : 0.0;
      for (int m = 0; m < r_b; ++m) s -= UB[(size_t)i * r_b + m] * std::conj(UB[(size_t)j * r_b + m]);
      FB[(size_t)i * q + j] = s;
    }
  if (filter == 0) {
    for (int i = 0; i < p; ++i)  // P = FA (x) FB
      for (int j = 0; j < q; ++j)
        for (int k = 0; k < p; ++k)
          for (int l = 0; l < q; ++l)
            P[(size_t)(i * q + j) * n + (k * q + l)] = FA[(size_t)i * p + k] * FB[(size_t)j * q + l];
  } else {
    // W[(i q + j), (ma r_b + mb)] = UA[i][ma] UB[j][mb];  P = I - W W^H
    const int nw = r_a * r_b;
    std::vector<cd> Wm((size_t)n * nw);
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < q; ++j)
        for (int ma = 0; ma < r_a; ++ma)
          for (int mb = 0; mb < r_b; ++mb)
            Wm[(size_t)(i * q + j) * nw + ma * r_b + mb] =
                UA[(size_t)i * r_a + ma] * UB[(size_t)j * r_b + mb];
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        cd s = (r == c) ? 1.0 : 0.0;
        for (int m = 0; m < nw; ++m) s -= Wm[(size_t)r * nw + m] * std::conj(Wm[(size_t)c * nw + m]);
        P[(size_t)r * n + c] = s;
      }
  }
  std::vector<cd> Px(n), d(n), Pd(n);
  for (int r = 0; r < n; ++r) {
    cd s = 0;
    for (int c = 0; c < n; ++c) s += P[(size_t)r * n + c] * x[c];
    Px[r] = s;
  }
  const double inv = 1.0 / std::sqrt(double(n));
  for (int v = 0; v < V; ++v) {
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < q; ++j)
        d[i * q + j] = bank_a[(size_t)v * p + i] * bank_b[(size_t)v * q + j] * inv;
    double dn = 0;
    for (int r = 0; r < n; ++r) dn += std::norm(d[r]);
    cd num = 0, den = 0;
    for (int r = 0; r < n; ++r) num += std::conj(d[r]) * Px[r];
    for (int r = 0; r < n; ++r) {
      cd s = 0;
      for (int c = 0; c < n; ++c) s += P[(size_t)r * n + c] * d[c];
      Pd[r] = s;
    }
    for (int r = 0; r < n; ++r) den += std::conj(d[r]) * Pd[r];
    const double dd = den.real();
    if (cond) cond[v] = (dn > 0) ? dd / dn : 0.0;
    T[v] = (dd < 1e-12 * dn) ? 0.0 : std::norm(num) / dd;
  }
}

inline cd ld(const float* base, size_t idx) { return cd(base[2 * idx], base[2 * idx + 1]); }

}  // namespace

extern "C" {

// O2: S (pq x pq, row-major, interleaved complex128) from n training
// snapshots X_m (n x p x q, interleaved complex128), x_m = vec(X_m^T).
void oracle_scm(const double* Xtr, int n, int p, int q, double* S_out) {
  const int pq = p * q;
  std::vector<cd> S((size_t)pq * pq, cd(0, 0));
  for (int m = 0; m < n; ++m) {
    const double* X = Xtr + (size_t)m * pq * 2;
    for (int r = 0; r < pq; ++r)
      for (int c = 0; c < pq; ++c) {
        cd xr(X[2 * r], X[2 * r + 1]), xc(X[2 * c], X[2 * c + 1]);
        S[(size_t)r * pq + c] += xr * std::conj(xc);
      }
  }
  for (size_t i = 0; i < S.size(); ++i) {
    S[i] /= double(n);
    S_out[2 * i] = S[i].real();
    S_out[2 * i + 1] = S[i].imag();
  }
}

// O3: Alg. 1.  S (pq x pq) -> R (p^2 x q^2), both row-major complex128.
void oracle_rearrange(const double* S_in, int p, int q, double* R_out) {
  const int pq = p * q;
  std::vector<cd> S((size_t)pq * pq), R;
  for (size_t i = 0; i < S.size(); ++i) S[i] = cd(S_in[2 * i], S_in[2 * i + 1]);
  rearrange_alg1(S, p, q, R);
  for (size_t i = 0; i < R.size(); ++i) {
    R_out[2 * i] = R[i].real();
    R_out[2 * i + 1] = R[i].imag();
  }
}

// Cyclic Jacobi eigendecomposition of a Hermitian n x n matrix (row-major
// complex128).  w: n eigenvalues (decreasing); U: n x n eigenvectors (columns).
void oracle_eigh(const double* M_in, int n, double* w_out, double* U_out) {
  std::vector<cd> M((size_t)n * n), U;
  for (size_t i = 0; i < M.size(); ++i) M[i] = cd(M_in[2 * i], M_in[2 * i + 1]);
  std::vector<double> w;
  jacobi_herm(M, n, w, U);
  for (int i = 0; i < n; ++i) w_out[i] = w[i];
  for (size_t i = 0; i < U.size(); ++i) {
    U_out[2 * i] = U[i].real();
    U_out[2 * i + 1] = U[i].imag();
  }
}

// O4-O6: Alg. 2 on a given S.  Outputs (complex128 interleaved, row-major):
// A (p x p), B (q x q), UA (p x r_a), UB (q x r_b); lamA (r_a), lamB (r_b),
// wB (q: all eigenvalues of herm(vec^-1 b) after trace normalisation),
// eta_hist (up to max_iter entries).  Any output may be null.  Returns the
// number of iterations.
int oracle_lrkron(const double* S_in, int p, int q, int r_a, int r_b, double eps, int max_iter,
                  double* A_out, double* B_out, double* UA_out, double* UB_out, double* lamA,
                  double* lamB, double* wB, double* eta_out, double* eta_hist) {
  const int pq = p * q;
  std::vector<cd> S((size_t)pq * pq);
  for (size_t i = 0; i < S.size(); ++i) S[i] = cd(S_in[2 * i], S_in[2 * i + 1]);
  LRKronResult r;
  lrkron(S, p, q, r_a, r_b, eps, max_iter, r);
  auto put = [](const std::vector<cd>& v, double* o) {
    if (!o) return;
    for (size_t i = 0; i < v.size(); ++i) {
      o[2 * i] = v[i].real();
      o[2 * i + 1] = v[i].imag();
    }
  };
  put(r.A, A_out);
  put(r.B, B_out);
  put(r.UA, UA_out);
  put(r.UB, UB_out);
  for (int m = 0; m < r_a && lamA; ++m) lamA[m] = r.lamA[m];
  for (int m = 0; m < r_b && lamB; ++m) lamB[m] = r.lamB[m];
  for (int m = 0; m < q && wB; ++m) wB[m] = r.wB_all[m];
  if (eta_out) *eta_out = r.eta;
  for (size_t m = 0; m < r.eta_hist.size() && eta_hist; ++m) eta_hist[m] = r.eta_hist[m];
  return r.iters;
}

// O7 on a given snapshot X (p x q complex128) and factors UA (p x r_a), UB
// (q x r_b).  bank_a (V x p), bank_b (V x q) complex128.  Outputs T (V) and
// cond (V) = d^H P d / |d|^2.
void oracle_stat(const double* X_in, const double* UA_in, const double* UB_in, int p, int q,
                 int r_a, int r_b, const double* ba_in, const double* bb_in, int V, double* T,
                 double* cond, int filter) {
  const int n = p * q;
  std::vector<cd> x(n), UA((size_t)p * r_a), UB((size_t)q * r_b), ba((size_t)V * p),
      bb((size_t)V * q);
  for (int i = 0; i < n; ++i) x[i] = cd(X_in[2 * i], X_in[2 * i + 1]);
  for (size_t i = 0; i < UA.size(); ++i) UA[i] = cd(UA_in[2 * i], UA_in[2 * i + 1]);
  for (size_t i = 0; i < UB.size(); ++i) UB[i] = cd(UB_in[2 * i], UB_in[2 * i + 1]);
  for (size_t i = 0; i < ba.size(); ++i) ba[i] = cd(ba_in[2 * i], ba_in[2 * i + 1]);
  for (size_t i = 0; i < bb.size(); ++i) bb[i] = cd(bb_in[2 * i], bb_in[2 * i + 1]);
  kstap_stat(x, UA, UB, p, q, r_a, r_b, ba, bb, V, T, cond, filter);
}

// Whole per-cell pipeline (O1-O7) over a list of cells of one frame.
//   Y: p x H_in x W_in complex64 (interleaved float pairs), row = range.
//   cells: flattened cell indices r * W + c, W = W_in - 2 Ra - q + 1.
// Outputs for listed cell k are written at offset k:
//   T_all[k*V + v], Tmax[k], vidx[k], map[k], cond[k*V + v],
//   PA[k] = U_A U_A^H (p x p complex128), PB[k] = U_B U_B^H (q x q complex128),
//   lamA[k*r_a..], lamB[k*r_b..], gapB[k] = (w_{r_b-1} - w_{r_b}) / w_0,
//   iters[k], eta[k].
// Any output pointer may be null.  Returns 0, or -1 on bad arguments.
int oracle_kstap_cells(const float* Y, int p, int H_in, int W_in, int q, int r_a, int r_b,
                       int Rr, int Ra, int Gr, int Ga, double eps, int max_iter,
                       const float* bank_a, const float* bank_b, int V, double tau,
                       const int64_t* cells, int64_t n_cells, double* T_all, double* Tmax,
                       int32_t* vidx, uint8_t* map, double* cond, double* PA, double* PB,
                       double* lamA, double* lamB, double* gapB, int32_t* iters, double* eta,
                       int nthreads, int filter) {
  const int H = H_in - 2 * Rr;
  const int W = W_in - 2 * Ra - q + 1;
  if (p < 1 || q < 2 || H < 1 || W < 1 || r_a < 1 || r_a > p || r_b < 1 || r_b >= q || V < 1)
    return -1;
  if (Gr > Rr || Ga > Ra || Gr < 0 || Ga < 0) return -1;
  const int pq = p * q;
  std::vector<cd> ba((size_t)V * p), bb((size_t)V * q);
  for (size_t i = 0; i < ba.size(); ++i) ba[i] = ld(bank_a, i);
  for (size_t i = 0; i < bb.size(); ++i) bb[i] = ld(bank_b, i);
  auto Yat = [&](int ch, int row, int col) -> cd {
    return ld(Y, ((size_t)ch * H_in + row) * W_in + col);
  };
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t k = 0; k < n_cells; ++k) {
    const int64_t cell = cells[k];
    if (cell < 0 || cell >= (int64_t)H * W) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      bad = 1;
      continue;
    }
    const int r = (int)(cell / W), c = (int)(cell % W);
    std::vector<cd> x(pq);  // O1
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < q; ++j) x[i * q + j] = Yat(i, r + Rr, c + Ra + j);
    std::vector<cd> S((size_t)pq * pq, cd(0, 0)), xm(pq);  // O2
    int n = 0;
    for (int dr = -Rr; dr <= Rr; ++dr)
      for (int dc = -Ra; dc <= Ra; ++dc) {
        if (std::abs(dr) <= Gr && std::abs(dc) <= Ga) continue;
        for (int i = 0; i < p; ++i)
          for (int j = 0; j < q; ++j) xm[i * q + j] = Yat(i, r + dr + Rr, c + dc + Ra + j);
        for (int a = 0; a < pq; ++a)
          for (int b2 = 0; b2 < pq; ++b2) S[(size_t)a * pq + b2] += xm[a] * std::conj(xm[b2]);
        ++n;
      }
    for (auto& s : S) s /= double(n);
    LRKronResult res;  // O3-O6
    lrkron(S, p, q, r_a, r_b, eps, max_iter, res);
    std::vector<double> T(V), cnd(V);  // O7
    kstap_stat(x, res.UA, res.UB, p, q, r_a, r_b, ba, bb, V, T.data(), cnd.data(), filter);
    double tm = -1;
    int vi = 0;
    for (int v = 0; v < V; ++v)
      if (T[v] > tm) {
        tm = T[v];
        vi = v;
      }
    if (T_all)
      for (int v = 0; v < V; ++v) T_all[k * V + v] = T[v];
    if (cond)
      for (int v = 0; v < V; ++v) cond[k * V + v] = cnd[v];
    if (Tmax) Tmax[k] = tm;
    if (vidx) vidx[k] = vi;
    if (map) map[k] = (tm > tau) ? 1 : 0;
    if (PA)
      for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
          cd s = 0;
          for (int m = 0; m < r_a; ++m)
            s += res.UA[(size_t)i * r_a + m] * std::conj(res.UA[(size_t)j * r_a + m]);
          const size_t o = ((size_t)k * p * p + (size_t)i * p + j) * 2;
          PA[o] = s.real();
          PA[o + 1] = s.imag();
        }
    if (PB)
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
          cd s = 0;
          for (int m = 0; m < r_b; ++m)
            s += res.UB[(size_t)i * r_b + m] * std::conj(res.UB[(size_t)j * r_b + m]);
          const size_t o = ((size_t)k * q * q + (size_t)i * q + j) * 2;
          PB[o] = s.real();
          PB[o + 1] = s.imag();
        }
    if (lamA)
      for (int m = 0; m < r_a; ++m) lamA[k * r_a + m] = res.lamA[m];
    if (lamB)
      for (int m = 0; m < r_b; ++m) lamB[k * r_b + m] = res.lamB[m];
    if (gapB)
      gapB[k] = (res.wB_all[0] != 0) ? (res.wB_all[r_b - 1] - res.wB_all[r_b]) / res.wB_all[0]
                                     : 0.0;
    if (iters) iters[k] = res.iters;
    if (eta) eta[k] = res.eta;
  }
  return bad ? -1 : 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
