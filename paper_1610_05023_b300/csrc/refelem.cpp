// Nodal reference elements (FP64, host).  Sec. 3.2: nodal DG of degree N on
// lines, triangles and tetrahedra with Warp & Blend tetrahedron nodes
// (Warburton 2006); triangle and line nodes coincide with the tetrahedron's
// face and edge nodes.  Elemental matrices: V (orthonormal modal basis at the
// nodes), D = V_r V^{-1}, M = (V V^T)^{-1}, LIFT = V V^T E (face mass blocks).
#include <algorithm>
#include <cmath>

#include "setup.h"

namespace dgh {

const int kSigma[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

Mat matmul(const Mat &A, const Mat &B) {
    Mat C(A.rows, B.cols);
    for (int i = 0; i < A.rows; ++i)
        for (int k = 0; k < A.cols; ++k) {
            const double a = A(i, k);
            if (a == 0.0) continue;
            for (int j = 0; j < B.cols; ++j) C(i, j) += a * B(k, j);
        }
    return C;
}

Mat transpose(const Mat &A) {
    Mat T(A.cols, A.rows);
    for (int i = 0; i < A.rows; ++i)
        for (int j = 0; j < A.cols; ++j) T(j, i) = A(i, j);
    return T;
}

bool invert(const Mat &A, Mat &Ainv) {
    const int n = A.rows;
    Mat W = A;
    Ainv = Mat(n, n);
    for (int i = 0; i < n; ++i) Ainv(i, i) = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(W(r, col)) > std::fabs(W(piv, col))) piv = r;
        if (std::fabs(W(piv, col)) < 1e-300) return false;
        if (piv != col)
            for (int j = 0; j < n; ++j) {
                std::swap(W(piv, j), W(col, j));
                std::swap(Ainv(piv, j), Ainv(col, j));
            }
        const double d = 1.0 / W(col, col);
        for (int j = 0; j < n; ++j) {
            W(col, j) *= d;
            Ainv(col, j) *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = W(r, col);
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                W(r, j) -= f * W(col, j);
                Ainv(r, j) -= f * Ainv(col, j);
            }
        }
    }
    return true;
}

// ------------------------------------------------------------------ Jacobi
// Classical Jacobi polynomial P_n^{(a,b)} by the three-term recurrence,
// normalised by its norm h_n = 2^{a+b+1} G(n+a+1) G(n+b+1) / ((2n+a+b+1) n! G(n+a+b+1)).
static double jacobi_classical(double x, double a, double b, int n) {
    if (n == 0) return 1.0;
    double p0 = 1.0;
    double p1 = 0.5 * (a - b + (a + b + 2.0) * x);
    for (int k = 2; k <= n; ++k) {
        const double s = 2.0 * k + a + b;
        const double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
        const double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
        const double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
        const double p2 = (c2 * p1 - c3 * p0) / c1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

static double jacobi_norm2(double a, double b, int n) {
    return std::exp((a + b + 1.0) * std::log(2.0) + std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) -
                    std::lgamma(n + 1.0) - std::lgamma(n + a + b + 1.0)) /
           (2.0 * n + a + b + 1.0);
}

static double jac(double x, double a, double b, int n) {
    return jacobi_classical(x, a, b, n) / std::sqrt(jacobi_norm2(a, b, n));
}

static double djac(double x, double a, double b, int n) {
    if (n == 0) return 0.0;
    return 0.5 * (n + a + b + 1.0) * jacobi_classical(x, a + 1.0, b + 1.0, n - 1) / std::sqrt(jacobi_norm2(a, b, n));
}

// GLL points: the ends and the roots of P_N' (Newton from the Chebyshev points).
std::vector<double> gll_points(int N) {
    std::vector<double> x(N + 1);
    x[0] = -1.0;
    x[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        double z = -std::cos(M_PI * j / N);
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < N; ++k) {
                const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_N, p0 = P_{N-1}
            const double d1 = N * (p0 - z * p1) / (1.0 - z * z);
            const double d2 = (2.0 * z * d1 - N * (N + 1.0) * p1) / (1.0 - z * z);
            const double dz = d1 / d2;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[j] = z;
    }
    std::sort(x.begin(), x.end());
    return x;
}

double warp_alpha_tet(int N) {
    static const double tab[15] = {0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577,
                                   1.1603, 1.10153, 0.6080, 0.4523, 0.8856, 0.8717, 0.9655};
    return N <= 15 ? tab[N - 1] : 1.0;
}

// ------------------------------------------------------------------ Warp & Blend
// Displacement of the equispaced 1D nodes onto the GLL nodes, interpolated in
// the equispaced Lagrange basis and divided by the blend 1 - x^2.
static double divided_warp(int N, const std::vector<double> &xg, double x) {
    if (std::fabs(x) >= 1.0 - 1e-10) return 0.0;
    double w = 0.0;
    for (int i = 0; i <= N; ++i) {
        const double xi = -1.0 + 2.0 * i / N;
        double l = 1.0;
        for (int j = 0; j <= N; ++j)
            if (j != i) l *= (x - (-1.0 + 2.0 * j / N)) / (xi - (-1.0 + 2.0 * j / N));
        w += (xg[i] - xi) * l;
    }
    return w / (1.0 - x * x);
}

// Warp of an equilateral triangle with barycentrics (top, left, right); the
// result is expressed in the frame (left->right, upward).
static void tri_warp(int N, double alpha, const std::vector<double> &xg, double top, double left, double right,
                     double &dx, double &dy) {
    const double w1 = 4.0 * left * right * divided_warp(N, xg, right - left) * (1.0 + alpha * alpha * top * top);
    const double w2 = 4.0 * top * right * divided_warp(N, xg, top - right) * (1.0 + alpha * alpha * left * left);
    const double w3 = 4.0 * top * left * divided_warp(N, xg, left - top) * (1.0 + alpha * alpha * right * right);
    const double c2 = std::cos(2.0 * M_PI / 3.0), s2 = std::sin(2.0 * M_PI / 3.0);
    const double c3 = std::cos(4.0 * M_PI / 3.0), s3 = std::sin(4.0 * M_PI / 3.0);
    dx = w1 + c2 * w2 + c3 * w3;
    dy = s2 * w2 + s3 * w3;
}

static void tri_nodes(int N, double alpha, std::vector<double> &r, std::vector<double> &s) {
    const std::vector<double> xg = gll_points(N);
    r.clear();
    s.clear();
    const double q3 = std::sqrt(3.0);
    for (int j = 0; j <= N; ++j)
        for (int i = 0; i <= N - j; ++i) {
            const double top = double(j) / N, right = double(i) / N, left = 1.0 - top - right;
            double X = right - left, Y = (2.0 * top - left - right) / q3;
            double dx, dy;
            tri_warp(N, alpha, xg, top, left, right, dx, dy);
            X += dx;
            Y += dy;
            const double T = (q3 * Y + 1.0) / 3.0;
            const double R = (3.0 * X - q3 * Y + 2.0) / 6.0;
            r.push_back(2.0 * R - 1.0);
            s.push_back(2.0 * T - 1.0);
        }
}

static void tet_nodes(int N, std::vector<double> &r, std::vector<double> &s, std::vector<double> &t) {
    const std::vector<double> xg = gll_points(N);
    const double alpha = warp_alpha_tet(N);
    const double q3 = std::sqrt(3.0), q6 = std::sqrt(6.0);
    // equilateral vertices of the reference vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1)
    const double E[4][3] = {{-1.0, -1.0 / q3, -1.0 / q6}, {1.0, -1.0 / q3, -1.0 / q6},
                            {0.0, 2.0 / q3, -1.0 / q6}, {0.0, 0.0, 3.0 / q6}};
    // face f = zero set of barycentric la; its triangle: top lb, left lc, right ld
    const int FT[4][4] = {{3, 2, 0, 1}, {2, 3, 0, 1}, {0, 3, 1, 2}, {1, 3, 0, 2}};
    const double tol = 1e-10;
    r.clear();
    s.clear();
    t.clear();
    for (int k = 0; k <= N; ++k)
        for (int j = 0; j <= N - k; ++j)
            for (int i = 0; i <= N - k - j; ++i) {
                const double re = -1.0 + 2.0 * i / N, se = -1.0 + 2.0 * j / N, te = -1.0 + 2.0 * k / N;
                double L[4] = {-(1.0 + re + se + te) / 2.0, (1.0 + re) / 2.0, (1.0 + se) / 2.0, (1.0 + te) / 2.0};
                double X[3] = {0, 0, 0};
                for (int v = 0; v < 4; ++v)
                    for (int d = 0; d < 3; ++d) X[d] += L[v] * E[v][d];
                double sh[3] = {0, 0, 0};
                for (int f = 0; f < 4; ++f) {
                    const int la = FT[f][0], lb = FT[f][1], lc = FT[f][2], ld = FT[f][3];
                    double e1[3], e2[3], n1 = 0, n2 = 0;
                    for (int d = 0; d < 3; ++d) {
                        e1[d] = E[ld][d] - E[lc][d];
                        e2[d] = E[lb][d] - 0.5 * (E[lc][d] + E[ld][d]);
                        n1 += e1[d] * e1[d];
                        n2 += e2[d] * e2[d];
                    }
                    n1 = std::sqrt(n1);
                    n2 = std::sqrt(n2);
                    double dx, dy;
                    tri_warp(N, alpha, xg, L[lb], L[lc], L[ld], dx, dy);
                    double blend = L[lb] * L[lc] * L[ld];
                    const double den = (L[lb] + 0.5 * L[la]) * (L[lc] + 0.5 * L[la]) * (L[ld] + 0.5 * L[la]);
                    if (den > tol) blend = (1.0 + alpha * alpha * L[la] * L[la]) * blend / den;
                    const int npos = (L[lb] > tol) + (L[lc] > tol) + (L[ld] > tol);
                    if (L[la] < tol && npos < 3) {
                        for (int d = 0; d < 3; ++d) sh[d] = dx * e1[d] / n1 + dy * e2[d] / n2;
                    } else {
                        for (int d = 0; d < 3; ++d) sh[d] += blend * (dx * e1[d] / n1 + dy * e2[d] / n2);
                    }
                }
                for (int d = 0; d < 3; ++d) X[d] += sh[d];
                // invert X = sum_v L_v E_v with sum L = 1
                Mat A(3, 3);
                double rhs[3];
                for (int d = 0; d < 3; ++d) {
                    A(d, 0) = 0.5 * (E[1][d] - E[0][d]);
                    A(d, 1) = 0.5 * (E[2][d] - E[0][d]);
                    A(d, 2) = 0.5 * (E[3][d] - E[0][d]);
                    rhs[d] = X[d] - 0.5 * (E[1][d] + E[2][d] + E[3][d] - E[0][d]);
                }
                Mat Ai;
                invert(A, Ai);
                double rst[3] = {0, 0, 0};
                for (int a = 0; a < 3; ++a)
                    for (int d = 0; d < 3; ++d) rst[a] += Ai(a, d) * rhs[d];
                r.push_back(rst[0]);
                s.push_back(rst[1]);
                t.push_back(rst[2]);
            }
}

// ------------------------------------------------------------------ modal bases
// Triangle: psi_ij = sqrt2 P_i(a) P_j^{(2i+1,0)}(b) (1-b)^i, a = 2(1+r)/(1-s)-1, b = s.
static void tri_basis(double r, double s, int i, int j, double &f, double &fr, double &fs) {
    const double a = (std::fabs(1.0 - s) > 1e-12) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
    const double b = s;
    const double A = jac(a, 0, 0, i), dA = djac(a, 0, 0, i);
    const double B = jac(b, 2 * i + 1, 0, j), dB = djac(b, 2 * i + 1, 0, j);
    const double q = 1.0 - b;
    const double qi = std::pow(q, i), qim1 = i > 0 ? std::pow(q, i - 1) : 0.0;
    const double c = std::sqrt(2.0);
    f = c * A * B * qi;
    // d/dr = dA * da/dr * B q^i with da/dr = 2/(1-b)
    fr = c * 2.0 * dA * B * qim1;
    // d/ds: da/ds = (1+a)/(1-b), d/db[B q^i] = dB q^i - i B q^{i-1}
    fs = c * (dA * (1.0 + a) * B * qim1 + A * (dB * qi - i * B * qim1));
}

// Tetrahedron: psi_ijk = 2 sqrt2 P_i(a) P_j^{(2i+1,0)}(b)(1-b)^i P_k^{(2i+2j+2,0)}(c)(1-c)^{i+j}.
static void tet_basis(double r, double s, double t, int i, int j, int k, double &f, double &fr, double &fs,
                      double &ft) {
    const double a = (std::fabs(s + t) > 1e-12) ? 2.0 * (1.0 + r) / (-s - t) - 1.0 : -1.0;
    const double b = (std::fabs(1.0 - t) > 1e-12) ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0 : -1.0;
    const double c = t;
    const double A = jac(a, 0, 0, i), dA = djac(a, 0, 0, i);
    const double B = jac(b, 2 * i + 1, 0, j), dB = djac(b, 2 * i + 1, 0, j);
    const double C = jac(c, 2 * i + 2 * j + 2, 0, k), dC = djac(c, 2 * i + 2 * j + 2, 0, k);
    const double qb = 1.0 - b, qc = 1.0 - c;
    auto pw = [](double x, int e) { return e < 0 ? 0.0 : std::pow(x, e); };
    const double fac = 2.0 * std::sqrt(2.0);
    f = fac * A * B * pw(qb, i) * C * pw(qc, i + j);
    // chain rule with -s-t = (1-b)(1-c)/2:
    //  da/dr = 4/((1-b)(1-c)), da/ds = da/dt = 2(1+a)/((1-b)(1-c)),
    //  db/ds = 2/(1-c), db/dt = (1+b)/(1-c), dc/dt = 1
    const double Bb = dB * pw(qb, i) - i * B * pw(qb, i - 1);  // d/db [B (1-b)^i]
    const double Cc = dC * pw(qc, i + j) - (i + j) * C * pw(qc, i + j - 1);
    const double ta = dA * B * C * pw(qb, i - 1) * pw(qc, i + j - 1);
    fr = fac * 4.0 * ta;
    fs = fac * (2.0 * (1.0 + a) * ta + 2.0 * A * Bb * C * pw(qc, i + j - 1));
    ft = fac * (2.0 * (1.0 + a) * ta + (1.0 + b) * A * Bb * C * pw(qc, i + j - 1) + A * B * pw(qb, i) * Cc);
}

// ------------------------------------------------------------------ builders
void build_line(int N, RefLine &L) {
    L.N = N;
    L.Np = N + 1;
    L.r = gll_points(N);
    Mat V(L.Np, L.Np), Vr(L.Np, L.Np);
    for (int n = 0; n < L.Np; ++n)
        for (int j = 0; j < L.Np; ++j) {
            V(n, j) = jac(L.r[n], 0, 0, j);
            Vr(n, j) = djac(L.r[n], 0, 0, j);
        }
    Mat Vi;
    invert(V, Vi);
    L.V = V;
    L.Dr = matmul(Vr, Vi);
    Mat VVt = matmul(V, transpose(V));
    invert(VVt, L.M);
    Mat E(L.Np, 2);
    E(0, 0) = 1.0;
    E(N, 1) = 1.0;
    L.LIFT = matmul(VVt, E);
}

void build_tri(int N, double alpha, RefTri &T) {
    T.N = N;
    T.Np = (N + 1) * (N + 2) / 2;
    T.Nfp = N + 1;
    tri_nodes(N, alpha, T.r, T.s);
    Mat V(T.Np, T.Np), Vr(T.Np, T.Np), Vs(T.Np, T.Np);
    for (int n = 0; n < T.Np; ++n) {
        int col = 0;
        for (int i = 0; i <= N; ++i)
            for (int j = 0; j <= N - i; ++j, ++col) tri_basis(T.r[n], T.s[n], i, j, V(n, col), Vr(n, col), Vs(n, col));
    }
    Mat Vi;
    invert(V, Vi);
    T.V = V;
    T.Dr = matmul(Vr, Vi);
    T.Ds = matmul(Vs, Vi);
    Mat VVt = matmul(V, transpose(V));
    invert(VVt, T.M);
    T.Fmask.assign(3, {});
    for (int n = 0; n < T.Np; ++n) {
        if (std::fabs(T.s[n] + 1.0) < 1e-10) T.Fmask[0].push_back(n);
        if (std::fabs(T.r[n] + T.s[n]) < 1e-10) T.Fmask[1].push_back(n);
        if (std::fabs(T.r[n] + 1.0) < 1e-10) T.Fmask[2].push_back(n);
    }
    Mat E(T.Np, 3 * T.Nfp);
    for (int e = 0; e < 3; ++e) {
        Mat V1(T.Nfp, T.Nfp);
        for (int m = 0; m < T.Nfp; ++m) {
            const int n = T.Fmask[e][m];
            const double x = (e == 2) ? T.s[n] : T.r[n];
            for (int j = 0; j < T.Nfp; ++j) V1(m, j) = jac(x, 0, 0, j);
        }
        Mat Me, tmp = matmul(V1, transpose(V1));
        invert(tmp, Me);
        for (int m = 0; m < T.Nfp; ++m)
            for (int mm = 0; mm < T.Nfp; ++mm) E(T.Fmask[e][m], e * T.Nfp + mm) = Me(m, mm);
    }
    T.LIFT = matmul(VVt, E);
}

bool build_tet(int N, RefTet &T, std::string &err) {
    T.N = N;
    T.Np = (N + 1) * (N + 2) * (N + 3) / 6;
    T.Nfp = (N + 1) * (N + 2) / 2;
    tet_nodes(N, T.r, T.s, T.t);
    const int Np = T.Np;
    Mat V(Np, Np), Vr(Np, Np), Vs(Np, Np), Vt(Np, Np);
    for (int n = 0; n < Np; ++n) {
        int col = 0;
        for (int i = 0; i <= N; ++i)
            for (int j = 0; j <= N - i; ++j)
                for (int k = 0; k <= N - i - j; ++k, ++col)
                    tet_basis(T.r[n], T.s[n], T.t[n], i, j, k, V(n, col), Vr(n, col), Vs(n, col), Vt(n, col));
    }
    Mat Vi;
    if (!invert(V, Vi)) {
        err = "singular tetrahedron Vandermonde matrix";
        return false;
    }
    T.V = V;
    T.Dr = matmul(Vr, Vi);
    T.Ds = matmul(Vs, Vi);
    T.Dt = matmul(Vt, Vi);
    Mat VVt = matmul(V, transpose(V));
    invert(VVt, T.M);
    T.Fmask.assign(4, {});
    for (int n = 0; n < Np; ++n) {
        const double r = T.r[n], s = T.s[n], t = T.t[n];
        if (std::fabs(1.0 + t) < 1e-10) T.Fmask[0].push_back(n);
        if (std::fabs(1.0 + s) < 1e-10) T.Fmask[1].push_back(n);
        if (std::fabs(1.0 + r + s + t) < 1e-10) T.Fmask[2].push_back(n);
        if (std::fabs(1.0 + r) < 1e-10) T.Fmask[3].push_back(n);
    }
    for (int f = 0; f < 4; ++f)
        if ((int)T.Fmask[f].size() != T.Nfp) {
            err = "face node extraction failed";
            return false;
        }
    Mat E(Np, 4 * T.Nfp);
    std::vector<double> fa(T.Nfp), fb(T.Nfp);
    for (int f = 0; f < 4; ++f) {
        for (int m = 0; m < T.Nfp; ++m) {
            const int n = T.Fmask[f][m];
            fa[m] = (f <= 1) ? T.r[n] : T.s[n];
            fb[m] = (f == 0) ? T.s[n] : T.t[n];
        }
        Mat V2(T.Nfp, T.Nfp), dum1(T.Nfp, T.Nfp), dum2(T.Nfp, T.Nfp);
        for (int m = 0; m < T.Nfp; ++m) {
            int col = 0;
            for (int i = 0; i <= N; ++i)
                for (int j = 0; j <= N - i; ++j, ++col) tri_basis(fa[m], fb[m], i, j, V2(m, col), dum1(m, col), dum2(m, col));
        }
        Mat Mf, tmp = matmul(V2, transpose(V2));
        invert(tmp, Mf);
        for (int m = 0; m < T.Nfp; ++m)
            for (int mm = 0; mm < T.Nfp; ++mm) E(T.Fmask[f][m], f * T.Nfp + mm) = Mf(m, mm);
        // face-node barycentrics (vertices of the face at (-1,-1), (1,-1), (-1,1))
        if (f == 0) {
            T.facePerm.assign(6, std::vector<int>(T.Nfp, -1));
            for (int sg = 0; sg < 6; ++sg)
                for (int m = 0; m < T.Nfp; ++m) {
                    const double lam[3] = {-(fa[m] + fb[m]) / 2.0, (1.0 + fa[m]) / 2.0, (1.0 + fb[m]) / 2.0};
                    double mu[3];
                    for (int i = 0; i < 3; ++i) mu[kSigma[sg][i]] = lam[i];
                    for (int mm = 0; mm < T.Nfp; ++mm) {
                        const double l2[3] = {-(fa[mm] + fb[mm]) / 2.0, (1.0 + fa[mm]) / 2.0, (1.0 + fb[mm]) / 2.0};
                        if (std::fabs(l2[0] - mu[0]) + std::fabs(l2[1] - mu[1]) + std::fabs(l2[2] - mu[2]) < 1e-9) {
                            T.facePerm[sg][m] = mm;
                            break;
                        }
                    }
                    if (T.facePerm[sg][m] < 0) {
                        err = "face nodes are not symmetric";
                        return false;
                    }
                }
        }
    }
    T.LIFT = matmul(VVt, E);
    return true;
}

std::vector<double> tet_interp_row(const RefTet &T, double r, double s, double t) {
    // l(x)^T = psi(x)^T V^{-1}
    Mat Vi;
    invert(T.V, Vi);
    std::vector<double> psi(T.Np), out(T.Np, 0.0);
    int col = 0;
    for (int i = 0; i <= T.N; ++i)
        for (int j = 0; j <= T.N - i; ++j)
            for (int k = 0; k <= T.N - i - j; ++k, ++col) {
                double a, b, c, d;
                tet_basis(r, s, t, i, j, k, a, b, c, d);
                psi[col] = a;
            }
    for (int n = 0; n < T.Np; ++n)
        for (int m = 0; m < T.Np; ++m) out[n] += psi[m] * Vi(m, n);
    return out;
}

}  // namespace dgh
