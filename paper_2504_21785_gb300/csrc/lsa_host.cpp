// Host precomputation of the pseudo-inverse of the eps-free Gram matrix
// (Algorithm 2, Step 0; Remark 2).
//
// The Gram matrix of eq. 3.22 (paper convention, ones on the diagonal)
//   A~_jk = exp(-cq^2/4 (dq_j-dq_k)^2 - cp^2/4 (dp_j-dp_k)^2
//               + i cq cp/2 (dq_k-dq_j)(dp_j+dp_k))
// is Hermitian positive semi-definite, so its SVD is its eigen-decomposition.
// It is computed here by the cyclic complex Jacobi method in long double and
// rounded to double once; singular values below rcond * lambda_max are dropped.
// Keeping the factors (instead of the formed matrix A~^+) lets the device apply
// the pseudo-inverse as V (diag(1/lambda) (V^H f~)).
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace fgr {

namespace {
using cld = std::complex<long double>;

void jacobi_hermitian(int n, std::vector<cld> &A, std::vector<cld> &V) {
    V.assign(n * n, cld(0));
    for (int i = 0; i < n; ++i) V[i * n + i] = 1;
    for (int sweep = 0; sweep < 100; ++sweep) {
        long double off = 0, diag = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (i == j)
                    diag += std::norm(A[i * n + j]);
                else
                    off += std::norm(A[i * n + j]);
            }
        if (off <= 1e-40L * diag) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                cld apq = A[p * n + q];
                long double mag = std::abs(apq);
                if (mag == 0) continue;
                long double app = A[p * n + p].real(), aqq = A[q * n + q].real();
                // rotation J = [[c, s e], [-s conj(e), c]] on columns p, q with e = apq/|apq|
                cld e = apq / mag;
                long double tau = (aqq - app) / (2 * mag);
                long double t = (tau >= 0 ? 1 : -1) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
                long double c = 1 / std::sqrt(1 + t * t), s = t * c;
                // A <- J^H A J
                for (int k = 0; k < n; ++k) {  // columns
                    cld akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * std::conj(e) * akq;
                    A[k * n + q] = s * e * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows
                    cld apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * e * aqk;
                    A[q * n + k] = s * std::conj(e) * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    cld vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * std::conj(e) * vkq;
                    V[k * n + q] = s * e * vkp + c * vkq;
                }
            }
    }
}
}  // namespace

bool build_lsa(double cq, double cp, int nq, int np, double rcond, Lsa *out) {
    static const int s2[2] = {0, 1}, s4[4] = {-1, 0, 1, 2};
    if ((nq != 2 && nq != 4) || (np != 2 && np != 4) || !(cq > 0) || !(cp > 0)) return false;
    const int *sq = nq == 2 ? s2 : s4, *sp = np == 2 ? s2 : s4;
    Lsa L;
    L.nq = nq;
    L.np = np;
    L.n1 = nq * np;
    L.cq = cq;
    L.cp = cp;
    const int n = L.n1;
    for (int iq = 0; iq < nq; ++iq)
        for (int ip = 0; ip < np; ++ip) {
            L.dq[iq * np + ip] = sq[iq];
            L.dp[iq * np + ip] = sp[ip];
        }
    std::vector<cld> A(n * n), V;
    const long double lcq = cq, lcp = cp;
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
            long double ddq = L.dq[j] - L.dq[k], ddp = L.dp[j] - L.dp[k];
            long double re = -lcq * lcq / 4 * ddq * ddq - lcp * lcp / 4 * ddp * ddp;
            long double im = lcq * lcp / 2 * (L.dq[k] - L.dq[j]) * (L.dp[j] + L.dp[k]);
            A[j * n + k] = std::exp(re) * cld(std::cos(im), std::sin(im));
        }
    jacobi_hermitian(n, A, V);
    // sort eigenpairs by eigenvalue, descending
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (A[idx[j] * n + idx[j]].real() > A[idx[i] * n + idx[i]].real()) std::swap(idx[i], idx[j]);
    const long double lmax = A[idx[0] * n + idx[0]].real();
    L.rank = 0;
    for (int i = 0; i < n; ++i) {
        long double lam = A[idx[i] * n + idx[i]].real();
        L.lam[i] = (double)lam;
        if (lam > (long double)rcond * lmax) {
            L.inv_lam[i] = (double)(1.0L / lam);
            ++L.rank;
        } else {
            L.inv_lam[i] = 0.0;
        }
        for (int j = 0; j < n; ++j) {
            L.vr[j * kMaxN1 + i] = (double)V[j * n + idx[i]].real();
            L.vi[j * kMaxN1 + i] = (double)V[j * n + idx[i]].imag();
        }
    }
    // Chebyshev surrogate (used by the FP32 path): values of the true
    // coefficients at kCheb x kCheb Chebyshev nodes, then the discrete
    // Chebyshev transform.  Same eigen factors and cut-off as the FP64 path.
    const long double PI = 3.141592653589793238462643383279502884L;
    std::vector<long double> vbuf((size_t)kCheb * kCheb * kMaxN1 * 2);
    auto vals = [&](int ia, int ib, int k, int c) -> long double & {
        return vbuf[(((size_t)ia * kCheb + ib) * kMaxN1 + k) * 2 + c];
    };
    long double node[kCheb];
    for (int a = 0; a < kCheb; ++a) node[a] = std::cos(PI * (a + 0.5L) / kCheb);
    for (int ia = 0; ia < kCheb; ++ia)
        for (int ib = 0; ib < kCheb; ++ib) {
            const long double s = 0.5L + 0.5L * node[ia], t = 0.5L + 0.5L * node[ib];
            cld f[kMaxN1], y[kMaxN1];
            for (int j = 0; j < n; ++j) {
                long double re = -lcq * lcq / 4 * (L.dq[j] - s) * (L.dq[j] - s) -
                                 lcp * lcp / 4 * (L.dp[j] - t) * (L.dp[j] - t);
                long double im = lcq * lcp / 2 * (s - L.dq[j]) * (L.dp[j] + t);
                f[j] = std::exp(re) * cld(std::cos(im), std::sin(im));
            }
            for (int i = 0; i < n; ++i) {  // y = diag(inv_lam) V^H f
                cld acc = 0;
                for (int j = 0; j < n; ++j) acc += std::conj(V[j * n + idx[i]]) * f[j];
                long double lam = A[idx[i] * n + idx[i]].real();
                y[i] = lam > (long double)rcond * lmax ? acc / lam : cld(0);
            }
            for (int k = 0; k < n; ++k) {  // c~ = conj(V y)
                cld acc = 0;
                for (int i = 0; i < n; ++i) acc += V[k * n + idx[i]] * y[i];
                vals(ia, ib, k, 0) = acc.real();
                vals(ia, ib, k, 1) = -acc.imag();
            }
        }
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < kCheb; ++i)
            for (int j = 0; j < kCheb; ++j) {
                long double re = 0, im = 0;
                for (int ia = 0; ia < kCheb; ++ia)
                    for (int ib = 0; ib < kCheb; ++ib) {
                        long double w = std::cos(i * PI * (ia + 0.5L) / kCheb) *
                                        std::cos(j * PI * (ib + 0.5L) / kCheb);
                        re += w * vals(ia, ib, k, 0);
                        im += w * vals(ia, ib, k, 1);
                    }
                long double sc = 4.0L / (kCheb * kCheb);
                if (i == 0) sc *= 0.5L;
                if (j == 0) sc *= 0.5L;
                L.cheb_re[k][i][j] = (float)(re * sc);
                L.cheb_im[k][i][j] = (float)(im * sc);
            }
    *out = L;
    return true;
}

}  // namespace fgr
