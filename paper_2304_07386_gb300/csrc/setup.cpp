// Host-side setup of the SMM solver (see setup.hpp).
//
// Discretization (paper Secs. "Finite Element Preliminaries", "Transport
// Discretization", "Discrete Second Moment Methods"):
//  * mesh map x(xi) = sum_k x_k l_k(xi) on (m+1)^2 Gauss-Lobatto control
//    points; F = dx/dxi, J = det F, grad u = F^{-T} grad_hat u;
//  * DG space Y_p with a nodal basis on (p+1)^2 Gauss-Lobatto points;
//  * Gauss-Legendre quadrature with p+m+1 points per direction in volume
//    and on faces;
//  * upwind DG S_N local operator A_{K,d} = sigma_t M - Omega_x Gx - Omega_y Gy
//    + sum_{outflow faces} (Omega_x Fx_f + Omega_y Fy_f), with
//    M_ij = int phi_i phi_j, Gx_ij = int phi_j dphi_i/dx and the face
//    matrices F_f[a][b] = sum_q (n ds w)_q l_a(s_q) l_b(s_q) on the p+1 face
//    nodal points.  A face must have one sign of Omega.n over all its
//    quadrature points (checked);
//  * IP-SMM (Eq. ipsmm) element and face blocks with D = 1/(3 sigma_t),
//    kappa = kappa_scale {(p+1)^2/(sigma_t h)}, h_K = |K| / longest face of K.
#include "setup.hpp"

#include <algorithm>
#include <cstdint>
#include <array>
#include <cmath>
#include <cstring>
#include <unordered_map>

namespace smm {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Legendre P_k(x) and P_{k-1}(x) by the three-term recurrence.
void legendre(int k, double x, double& pk, double& pkm1) {
    double p0 = 1.0, p1 = x;
    if (k == 0) { pk = 1.0; pkm1 = 0.0; return; }
    for (int j = 2; j <= k; ++j) {
        double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    pk = p1;
    pkm1 = p0;
}

struct Lag1D {
    std::vector<double> nodes;
    // values and derivatives of all basis polynomials at x
    void eval(double x, double* v, double* d) const {
        const int k = (int)nodes.size();
        for (int a = 0; a < k; ++a) {
            double val = 1.0;
            for (int b = 0; b < k; ++b)
                if (b != a) val *= (x - nodes[b]) / (nodes[a] - nodes[b]);
            v[a] = val;
            double der = 0.0;
            for (int c = 0; c < k; ++c) {
                if (c == a) continue;
                double t = 1.0 / (nodes[a] - nodes[c]);
                for (int b = 0; b < k; ++b)
                    if (b != a && b != c) t *= (x - nodes[b]) / (nodes[a] - nodes[b]);
                der += t;
            }
            d[a] = der;
        }
    }
};

// Tensor basis values V[n] and reference gradients G[n][2] at (xi, eta).
void tensor_eval(const Lag1D& L, double xi, double eta, double* V, double* G) {
    const int k = (int)L.nodes.size();
    double vx[16], dx[16], vy[16], dy[16];
    L.eval(xi, vx, dx);
    L.eval(eta, vy, dy);
    for (int iy = 0; iy < k; ++iy)
        for (int ix = 0; ix < k; ++ix) {
            int i = iy * k + ix;
            V[i] = vx[ix] * vy[iy];
            G[2 * i] = dx[ix] * vy[iy];
            G[2 * i + 1] = vx[ix] * dy[iy];
        }
}

void face_ref(int f, double s, double& xi, double& eta) {
    switch (f) {
        case 0: xi = s; eta = 0.0; break;
        case 1: xi = 1.0; eta = s; break;
        case 2: xi = s; eta = 1.0; break;
        default: xi = 0.0; eta = s; break;
    }
}

int face_node(int p, int f, int a) {
    const int q = p + 1;
    switch (f) {
        case 0: return a;
        case 1: return a * q + p;
        case 2: return p * q + a;
        default: return a * q;
    }
}

void face_corner_ids(int m, int f, int& c0, int& c1) {
    const int q = m + 1;
    const int c00 = 0, c10 = m, c01 = m * q, c11 = m * q + m;
    switch (f) {
        case 0: c0 = c00; c1 = c10; break;
        case 1: c0 = c10; c1 = c11; break;
        case 2: c0 = c01; c1 = c11; break;
        default: c0 = c00; c1 = c01; break;
    }
}

// Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix.
bool invert(int n, const double* A, double* Ainv) {
    std::vector<double> a(A, A + n * n), b(n * n, 0.0);
    for (int i = 0; i < n; ++i) b[i * n + i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(a[i * n + k]) > std::fabs(a[piv * n + k])) piv = i;
        if (a[piv * n + k] == 0.0) return false;
        if (piv != k)
            for (int j = 0; j < n; ++j) {
                std::swap(a[k * n + j], a[piv * n + j]);
                std::swap(b[k * n + j], b[piv * n + j]);
            }
        double inv = 1.0 / a[k * n + k];
        for (int j = 0; j < n; ++j) { a[k * n + j] *= inv; b[k * n + j] *= inv; }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            double l = a[i * n + k];
            if (l == 0.0) continue;
            for (int j = 0; j < n; ++j) { a[i * n + j] -= l * a[k * n + j]; b[i * n + j] -= l * b[k * n + j]; }
        }
    }
    std::memcpy(Ainv, b.data(), sizeof(double) * n * n);
    return true;
}

// Per-element geometry at one reference point: physical point, F, J.
struct Geo {
    double x, y, F[4], J;   // F = [[dx/dxi, dx/deta], [dy/dxi, dy/deta]]
};

Geo map_point(const Lag1D& Lm, const double* ctrl, double xi, double eta) {
    const int k = (int)Lm.nodes.size();
    double vx[16], dx[16], vy[16], dy[16];
    Lm.eval(xi, vx, dx);
    Lm.eval(eta, vy, dy);
    Geo g{};
    for (int iy = 0; iy < k; ++iy)
        for (int ix = 0; ix < k; ++ix) {
            const double* c = ctrl + 2 * (iy * k + ix);
            double v = vx[ix] * vy[iy], gx = dx[ix] * vy[iy], gy = vx[ix] * dy[iy];
            g.x += c[0] * v;
            g.y += c[1] * v;
            g.F[0] += c[0] * gx;
            g.F[1] += c[0] * gy;
            g.F[2] += c[1] * gx;
            g.F[3] += c[1] * gy;
        }
    g.J = g.F[0] * g.F[3] - g.F[1] * g.F[2];
    return g;
}

// physical gradient = F^{-T} grad_hat
inline void phys_grad(const Geo& g, double gx_hat, double gy_hat, double& gx, double& gy) {
    // F^{-1} = 1/J [[F3, -F1], [-F2, F0]];  F^{-T} = 1/J [[F3, -F2], [-F1, F0]]
    gx = (g.F[3] * gx_hat - g.F[2] * gy_hat) / g.J;
    gy = (-g.F[1] * gx_hat + g.F[0] * gy_hat) / g.J;
}

// Face data of one element face at the face Gauss points.
struct FaceData {
    std::vector<double> V;    // [nfq][n]
    std::vector<double> G;    // [nfq][n][2]
    std::vector<double> nds;  // [nfq][2]
    double length = 0.0;
};

// Factor every neighbour block of the moment operator through the face data
// of the two elements.  With nodal Gauss-Lobatto bases the trace of u on a
// face is its p+1 face-node values, and the physical gradient there depends
// only on the trace and on the reference normal derivative, whose values at
// the face nodes are sum_t l'_t(0) u(line t).  So Aoff = E_f^T C E_f2 with a
// 2(p+1) x 2(p+1) matrix C, computed here as R_f^T Aoff R_f2 from right
// inverses (E R = I) and checked by rebuilding Aoff.
int factor_face_blocks(Setup& s, std::string& err) {
    const int n = s.n, p = s.p, p1 = s.p1, G = 2 * p1, ne = s.ne;
    Lag1D L;
    L.nodes = gauss_lobatto01(p1).x;
    std::vector<double> v(p1), d(p1);
    L.eval(0.0, v.data(), d.data());
    s.wd.assign(d.begin(), d.end());
    if (std::fabs(s.wd[1]) < 1e-12) { err = "degenerate face derivative"; return 4; }
    // R_f columns: trace a -> e_(a,0) - wd0/wd1 e_(a,1); derivative a -> e_(a,1) / wd1
    auto rcols = [&](int f, std::vector<double>& R) {  // R [n][G]
        R.assign((size_t)n * G, 0.0);
        for (int a = 0; a < p1; ++a) {
            const int n0 = face_line_node(p, f, a, 0), n1 = face_line_node(p, f, a, 1);
            R[(size_t)n0 * G + a] = 1.0;
            R[(size_t)n1 * G + a] = -s.wd[0] / s.wd[1];
            R[(size_t)n1 * G + p1 + a] = 1.0 / s.wd[1];
        }
    };
    std::vector<double> Rf[4];
    for (int f = 0; f < 4; ++f) rcols(f, Rf[f]);
    s.Cface.assign((size_t)ne * 4 * G * G, 0.0);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int e = 0; e < ne; ++e) {
        std::vector<double> T((size_t)n * G), Rb((size_t)n * n);
        for (int f = 0; f < 4; ++f) {
            if (s.nbr[e * 4 + f] < 0) continue;
            const int f2 = s.nbr_face[e * 4 + f];
            const double* A = &s.Aoff[((size_t)e * 4 + f) * n * n];
            const std::vector<double>& R1 = Rf[f];
            const std::vector<double>& R2 = Rf[f2];
            double* C = &s.Cface[((size_t)e * 4 + f) * G * G];
            // T = A R2 (n x G); C = R1^T T
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < G; ++c) {
                    double acc = 0.0;
                    for (int j = 0; j < n; ++j) acc += A[(size_t)i * n + j] * R2[(size_t)j * G + c];
                    T[(size_t)i * G + c] = acc;
                }
            for (int r = 0; r < G; ++r)
                for (int c = 0; c < G; ++c) {
                    double acc = 0.0;
                    for (int i = 0; i < n; ++i) acc += R1[(size_t)i * G + r] * T[(size_t)i * G + c];
                    C[r * G + c] = acc;
                }
            // rebuild E_f^T C E_f2 and compare
            std::fill(Rb.begin(), Rb.end(), 0.0);
            for (int r = 0; r < G; ++r)
                for (int c = 0; c < G; ++c) {
                    const double cv = C[r * G + c];
                    if (cv == 0.0) continue;
                    const int a = r % p1, b = c % p1;
                    for (int t = 0; t < p1; ++t) {
                        if (r < p1 && t > 0) break;
                        const double er = r < p1 ? 1.0 : s.wd[t];
                        const int ni = face_line_node(p, f, a, t);
                        for (int u = 0; u < p1; ++u) {
                            if (c < p1 && u > 0) break;
                            const double ec = c < p1 ? 1.0 : s.wd[u];
                            Rb[(size_t)ni * n + face_line_node(p, f2, b, u)] += er * cv * ec;
                        }
                    }
                }
            double amax = 0.0, dmax = 0.0;
            for (size_t ij = 0; ij < (size_t)n * n; ++ij) {
                amax = std::max(amax, std::fabs(A[ij]));
                dmax = std::max(dmax, std::fabs(A[ij] - Rb[ij]));
            }
            if (dmax > 1e-11 * amax) bad += 1;
        }
    }
    if (bad) { err = "neighbour block of the moment operator is not face-factorable"; return 4; }
    return 0;
}

// Global node of every element node for the continuous space V_p: the
// element nodes of a face are joined with the matching nodes of the
// neighbour's face (union-find), ids numbered by first appearance.
void continuous_numbering(Setup& s) {
    const int ne = s.ne, n = s.n, p = s.p;
    std::vector<int32_t> parent((size_t)ne * n);
    for (size_t k = 0; k < parent.size(); ++k) parent[k] = (int32_t)k;
    auto find = [&](int32_t x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    for (int e = 0; e < ne; ++e)
        for (int f = 0; f < 4; ++f) {
            const int e2 = s.nbr[e * 4 + f];
            if (e2 < 0) continue;
            const int f2 = s.nbr_face[e * 4 + f], flip = s.nbr_flip[e * 4 + f];
            for (int a = 0; a <= p; ++a) {
                const int32_t r1 = find(e * n + face_node(p, f, a));
                const int32_t r2 = find(e2 * n + face_node(p, f2, flip ? p - a : a));
                if (r1 != r2) parent[std::max(r1, r2)] = std::min(r1, r2);
            }
        }
    s.gid.assign((size_t)ne * n, -1);
    std::vector<int32_t> id_of((size_t)ne * n, -1);
    int ng = 0;
    for (size_t k = 0; k < (size_t)ne * n; ++k) {
        const int32_t r = find((int32_t)k);
        if (id_of[r] < 0) id_of[r] = ng++;
        s.gid[k] = id_of[r];
    }
    s.nglob = ng;
    s.grp.assign((size_t)ng + 1, 0);
    for (size_t k = 0; k < s.gid.size(); ++k) s.grp[(size_t)s.gid[k] + 1] += 1;
    for (int g = 0; g < ng; ++g) s.grp[(size_t)g + 1] += s.grp[g];
    s.ginc.assign(s.gid.size(), 0);
    std::vector<int32_t> pos(s.grp.begin(), s.grp.end() - 1);
    for (size_t k = 0; k < s.gid.size(); ++k) s.ginc[pos[s.gid[k]]++] = (int32_t)k;
    s.gown.assign((size_t)ng, 0);
    for (int g = 0; g < ng; ++g) s.gown[g] = s.ginc[s.grp[g]];
}

}  // namespace

Rule1D gauss_legendre01(int n) {
    Rule1D r;
    r.x.resize(n);
    r.w.resize(n);
    for (int i = 0; i < n; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, pm;
            legendre(n, x, pn, pm);
            double dp = n * (x * pn - pm) / (x * x - 1.0);
            double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double pn, pm;
        legendre(n, x, pn, pm);
        double dp = n * (x * pn - pm) / (x * x - 1.0);
        r.x[n - 1 - i] = 0.5 * (x + 1.0);
        r.w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return r;
}

Rule1D gauss_lobatto01(int n) {
    // nodes: +-1 and the roots of P'_{N}, N = n-1; Newton on
    // f(x) = x P_N - P_{N-1} (zero exactly at those points, up to the factor
    // (1-x^2) P'_N / N), from Chebyshev-Gauss-Lobatto guesses.
    Rule1D r;
    r.x.resize(n);
    r.w.resize(n);
    const int N = n - 1;
    for (int i = 0; i < n; ++i) {
        double x = -std::cos(kPi * i / N);
        if (i != 0 && i != N) {
            for (int it = 0; it < 100; ++it) {
                double pn, pm;
                legendre(N, x, pn, pm);
                double f = x * pn - pm;
                double fp = n * pn;  // derivative of x P_N - P_{N-1} equals (N+1) P_N
                double dx = f / fp;
                x -= dx;
                if (std::fabs(dx) < 1e-16) break;
            }
        }
        double pn, pm;
        legendre(N, x, pn, pm);
        r.x[i] = 0.5 * (x + 1.0);
        r.w[i] = 0.5 * 2.0 / (N * (N + 1.0) * pn * pn);
    }
    r.x[0] = 0.0;
    r.x[N] = 1.0;
    return r;
}

bool level_symmetric(int N, Quadrature& q) {
    double mu1;
    switch (N) {
        case 2: mu1 = 1.0 / std::sqrt(3.0); break;
        case 4: mu1 = std::sqrt((4.0 - std::sqrt(6.4)) / 12.0); break;  // fixed by the mu^4 condition
        case 6: mu1 = 0.2666355; break;
        case 8: mu1 = 0.2182179; break;
        case 10: mu1 = 0.1893213; break;
        case 12: mu1 = 0.1672126; break;
        default: return false;
    }
    const int L = N / 2;
    std::vector<double> mu(L);
    const double step = (N > 2) ? 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2) : 0.0;
    for (int i = 0; i < L; ++i) mu[i] = std::sqrt(mu1 * mu1 + i * step);
    struct Pt { int i, j, k, cls; };
    std::vector<Pt> pts;
    std::vector<std::array<int, 3>> classes;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L - i; ++j) {
            int k = L - 1 - i - j;
            std::array<int, 3> c{i, j, k};
            std::sort(c.begin(), c.end());
            int id = -1;
            for (size_t t = 0; t < classes.size(); ++t)
                if (classes[t] == c) id = (int)t;
            if (id < 0) { id = (int)classes.size(); classes.push_back(c); }
            pts.push_back({i, j, k, id});
        }
    // class weights from the even-moment conditions sum w mu^{2k} = 1/(2k+1),
    // k in {0, 2, 3, ..., nc}; solved by Gaussian elimination with pivoting
    const int nc = (int)classes.size();
    std::vector<double> A(nc * nc, 0.0), rhs(nc);
    for (int r = 0; r < nc; ++r) {
        int k = (r == 0) ? 0 : r + 1;
        for (const Pt& t : pts) A[r * nc + t.cls] += std::pow(mu[t.i], 2.0 * k);
        rhs[r] = 1.0 / (2.0 * k + 1.0);
    }
    std::vector<double> Ainv(nc * nc);
    if (!invert(nc, A.data(), Ainv.data())) return false;
    std::vector<double> wc(nc, 0.0);
    for (int r = 0; r < nc; ++r)
        for (int c = 0; c < nc; ++c) wc[r] += Ainv[r * nc + c] * rhs[c];
    const double sx[4] = {1, -1, -1, 1}, sy[4] = {1, 1, -1, -1};
    q.nd = 4 * (int)pts.size();
    q.ox.clear(); q.oy.clear(); q.w.clear();
    for (int quad = 0; quad < 4; ++quad)
        for (const Pt& t : pts) {
            q.ox.push_back(sx[quad] * mu[t.i]);
            q.oy.push_back(sy[quad] * mu[t.j]);
            q.w.push_back(2.0 * wc[t.cls] * (4.0 * kPi / 8.0));
        }
    return true;
}

int build_setup(const Input& in, Setup& s, std::string& err) {
    if (in.p < 1 || in.p > 4) { err = "p must be in 1..4"; return 1; }
    if (in.m < 1 || in.m > 6) { err = "geometry order must be in 1..6"; return 1; }
    if (in.ne <= 0 || !in.nodes || !in.elem_nodes || !in.sigma_t || !in.sigma_s || !in.q) {
        err = "missing mesh, cross sections or source";
        return 1;
    }
    if (!level_symmetric(in.sn, s.quad)) { err = "unsupported S_N order"; return 1; }
    s.ne = in.ne; s.m = in.m; s.p = in.p; s.p1 = in.p + 1; s.n = s.p1 * s.p1;
    s.nq = in.p + in.m + 1; s.nqv = s.nq * s.nq; s.nfq = s.nq; s.nd = s.quad.nd;
    const int ne = s.ne, n = s.n, p1 = s.p1, nd = s.nd, nfq = s.nfq, m1 = in.m + 1;
    const int nc = m1 * m1;
    // (element, ordinate) task ids e * nd + d, control point slots e * nc + k and
    // unknown ids e * n + i are 32-bit integers on the host and the device
    if ((long long)ne * std::max(std::max(nd, nc), n) > (long long)INT32_MAX) {
        err = "mesh too large: n_elem times the ordinates, control points or dofs per element exceeds 2^31 - 1";
        return 1;
    }
    for (int e = 0; e < ne; ++e) {
        if (!(in.sigma_t[e] > 0.0) || in.sigma_s[e] < 0.0 || in.sigma_s[e] > in.sigma_t[e]) {
            err = "need sigma_t > 0 and 0 <= sigma_s <= sigma_t";
            return 1;
        }
        for (int k = 0; k < nc; ++k) {
            int id = in.elem_nodes[e * nc + k];
            if (id < 0 || id >= in.n_nodes) { err = "control point id out of range"; return 1; }
        }
    }
    s.sigma_t.assign(in.sigma_t, in.sigma_t + ne);
    s.sigma_s.assign(in.sigma_s, in.sigma_s + ne);

    Lag1D Lp, Lm;
    Lp.nodes = gauss_lobatto01(p1).x;
    Lm.nodes = gauss_lobatto01(m1).x;
    const Rule1D gq = gauss_legendre01(s.nq);
    s.L1.resize(nfq * p1);
    {
        double d[16];
        for (int q = 0; q < nfq; ++q) Lp.eval(gq.x[q], &s.L1[q * p1], d);
    }

    // ---- connectivity from shared corner control points ----
    s.nbr.assign(ne * 4, -1);
    s.nbr_face.assign(ne * 4, -1);
    s.nbr_flip.assign(ne * 4, 0);
    {
        std::unordered_map<uint64_t, std::vector<int>> owner;
        owner.reserve(ne * 4);
        for (int e = 0; e < ne; ++e)
            for (int f = 0; f < 4; ++f) {
                int c0, c1;
                face_corner_ids(in.m, f, c0, c1);
                uint64_t a = (uint32_t)in.elem_nodes[e * nc + c0], b = (uint32_t)in.elem_nodes[e * nc + c1];
                if (a > b) std::swap(a, b);
                owner[(a << 32) | b].push_back(e * 4 + f);
            }
        for (auto& kv : owner) {
            auto& l = kv.second;
            if (l.size() > 2) { err = "face shared by more than two elements"; return 4; }
            if (l.size() == 2) {
                int e1 = l[0] / 4, f1 = l[0] % 4, e2 = l[1] / 4, f2 = l[1] % 4;
                int c0a, c1a, c0b, c1b;
                face_corner_ids(in.m, f1, c0a, c1a);
                face_corner_ids(in.m, f2, c0b, c1b);
                int flip = in.elem_nodes[e1 * nc + c0a] != in.elem_nodes[e2 * nc + c0b];
                s.nbr[e1 * 4 + f1] = e2; s.nbr_face[e1 * 4 + f1] = f2; s.nbr_flip[e1 * 4 + f1] = flip;
                s.nbr[e2 * 4 + f2] = e1; s.nbr_face[e2 * 4 + f2] = f1; s.nbr_flip[e2 * 4 + f2] = flip;
            }
        }
    }
    s.bface_id.assign(ne * 4, -1);
    s.bface_elem.clear(); s.bface_face.clear();
    for (int e = 0; e < ne; ++e)
        for (int f = 0; f < 4; ++f)
            if (s.nbr[e * 4 + f] < 0) {
                s.bface_id[e * 4 + f] = (int)s.bface_elem.size();
                s.bface_elem.push_back(e);
                s.bface_face.push_back(f);
            }
    s.nb = (int)s.bface_elem.size();

    // ---- per-element geometry, element matrices, face data ----
    s.M.assign((size_t)ne * n * n, 0.0);
    s.Gx.assign((size_t)ne * n * n, 0.0);
    s.Gy.assign((size_t)ne * n * n, 0.0);
    s.Kxx.assign((size_t)ne * n * n, 0.0);
    s.Ks.assign((size_t)ne * n * n, 0.0);
    s.Kyy.assign((size_t)ne * n * n, 0.0);
    s.Fx.assign((size_t)ne * 4 * p1 * p1, 0.0);
    s.Fy.assign((size_t)ne * 4 * p1 * p1, 0.0);
    s.Dfx.assign((size_t)ne * 4 * nfq * n, 0.0);
    s.Dfy.assign((size_t)ne * 4 * nfq * n, 0.0);
    s.nds.assign((size_t)ne * 4 * nfq * 2, 0.0);
    s.area.assign(ne, 0.0);
    s.hK.assign(ne, 0.0);
    std::vector<double> faceV((size_t)ne * 4 * nfq * n);  // basis values at face points
    std::vector<double> flen((size_t)ne * 4);
    int bad_jac = 0;

#pragma omp parallel for schedule(static) reduction(+ : bad_jac)
    for (int e = 0; e < ne; ++e) {
        double ctrl[2 * 64];
        for (int k = 0; k < nc; ++k) {
            int id = in.elem_nodes[e * nc + k];
            ctrl[2 * k] = in.nodes[2 * id];
            ctrl[2 * k + 1] = in.nodes[2 * id + 1];
        }
        std::vector<double> V(n), Gh(2 * n), G(2 * n);
        double* M = &s.M[(size_t)e * n * n];
        double* Gx = &s.Gx[(size_t)e * n * n];
        double* Gy = &s.Gy[(size_t)e * n * n];
        double* Kxx = &s.Kxx[(size_t)e * n * n];
        double* Ks = &s.Ks[(size_t)e * n * n];
        double* Kyy = &s.Kyy[(size_t)e * n * n];
        double area = 0.0;
        for (int qy = 0; qy < s.nq; ++qy)
            for (int qx = 0; qx < s.nq; ++qx) {
                Geo g = map_point(Lm, ctrl, gq.x[qx], gq.x[qy]);
                if (!(g.J > 0.0)) bad_jac += 1;
                double wJ = gq.w[qx] * gq.w[qy] * g.J;
                area += wJ;
                tensor_eval(Lp, gq.x[qx], gq.x[qy], V.data(), Gh.data());
                for (int i = 0; i < n; ++i) phys_grad(g, Gh[2 * i], Gh[2 * i + 1], G[2 * i], G[2 * i + 1]);
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) {
                        size_t ij = (size_t)i * n + j;
                        M[ij] += wJ * V[i] * V[j];
                        Gx[ij] += wJ * G[2 * i] * V[j];
                        Gy[ij] += wJ * G[2 * i + 1] * V[j];
                        Kxx[ij] += wJ * G[2 * i] * G[2 * j];
                        Ks[ij] += wJ * (G[2 * i] * G[2 * j + 1] + G[2 * i + 1] * G[2 * j]);
                        Kyy[ij] += wJ * G[2 * i + 1] * G[2 * j + 1];
                    }
            }
        s.area[e] = area;
        double longest = 0.0;
        for (int f = 0; f < 4; ++f) {
            double len = 0.0;
            for (int q = 0; q < nfq; ++q) {
                double xi, eta;
                face_ref(f, gq.x[q], xi, eta);
                Geo g = map_point(Lm, ctrl, xi, eta);
                if (!(g.J > 0.0)) bad_jac += 1;
                double tx, ty;
                if (f == 0 || f == 2) { tx = g.F[0]; ty = g.F[2]; } else { tx = g.F[1]; ty = g.F[3]; }
                double nx, ny;
                if (f == 0 || f == 1) { nx = ty; ny = -tx; } else { nx = -ty; ny = tx; }
                nx *= gq.w[q];
                ny *= gq.w[q];
                double* nds = &s.nds[(((size_t)e * 4 + f) * nfq + q) * 2];
                nds[0] = nx;
                nds[1] = ny;
                len += std::sqrt(nx * nx + ny * ny);
                tensor_eval(Lp, xi, eta, V.data(), Gh.data());
                for (int i = 0; i < n; ++i) {
                    double gx, gy;
                    phys_grad(g, Gh[2 * i], Gh[2 * i + 1], gx, gy);
                    s.Dfx[(((size_t)e * 4 + f) * nfq + q) * n + i] = gx;
                    s.Dfy[(((size_t)e * 4 + f) * nfq + q) * n + i] = gy;
                    faceV[(((size_t)e * 4 + f) * nfq + q) * n + i] = V[i];
                }
                for (int a = 0; a < p1; ++a)
                    for (int b = 0; b < p1; ++b) {
                        double lab = s.L1[q * p1 + a] * s.L1[q * p1 + b];
                        s.Fx[(((size_t)e * 4 + f) * p1 + a) * p1 + b] += nx * lab;
                        s.Fy[(((size_t)e * 4 + f) * p1 + a) * p1 + b] += ny * lab;
                    }
            }
            flen[e * 4 + f] = len;
            longest = std::max(longest, len);
        }
        s.hK[e] = area / longest;
    }
    if (bad_jac) { err = "non-positive Jacobian at a quadrature point"; return 4; }

    // ---- face direction per (e, d, f): 1 outflow, -1 inflow, 2 inflow at some
    //      quadrature points and outflow at others (mixed), 0 tangential ----
    s.fdir.assign((size_t)ne * nd * 4, 0);
    int64_t mixed = 0;
#pragma omp parallel for schedule(static) reduction(+ : mixed)
    for (int e = 0; e < ne; ++e)
        for (int d = 0; d < nd; ++d)
            for (int f = 0; f < 4; ++f) {
                bool pos = false, neg = false;
                for (int q = 0; q < nfq; ++q) {
                    const double* nds = &s.nds[(((size_t)e * 4 + f) * nfq + q) * 2];
                    double a = s.quad.ox[d] * nds[0] + s.quad.oy[d] * nds[1];
                    pos |= a > 0.0;
                    neg |= a < 0.0;
                }
                if (pos && neg) mixed += 1;
                s.fdir[((size_t)e * nd + d) * 4 + f] = pos && neg ? 2 : (pos ? 1 : (neg ? -1 : 0));
            }
    if (mixed && !in.lag_cycles) {
        err = "a face is inflow at some quadrature points and outflow at others for some ordinate";
        return 5;
    }
    // pointwise face matrices of the mixed faces: their outflow part enters the
    // local operator, their inflow part multiplies the upwind trace
    s.n_mixed = mixed;
    s.fmix_id.clear();
    s.fmix.clear();
    if (mixed) {
        s.fmix_id.assign((size_t)ne * nd * 4, -1);
        int32_t next = 0;
        for (size_t k = 0; k < s.fdir.size(); ++k)
            if (s.fdir[k] == 2) s.fmix_id[k] = next++;
        s.fmix.assign((size_t)next * 2 * p1 * p1, 0.0);
#pragma omp parallel for schedule(static)
        for (int e = 0; e < ne; ++e)
            for (int d = 0; d < nd; ++d)
                for (int f = 0; f < 4; ++f) {
                    const int32_t id = s.fmix_id[((size_t)e * nd + d) * 4 + f];
                    if (id < 0) continue;
                    double* fp = &s.fmix[(size_t)id * 2 * p1 * p1];
                    double* fn = fp + p1 * p1;
                    for (int q = 0; q < nfq; ++q) {
                        const double* nds = &s.nds[(((size_t)e * 4 + f) * nfq + q) * 2];
                        const double a = s.quad.ox[d] * nds[0] + s.quad.oy[d] * nds[1];
                        for (int i = 0; i < p1; ++i)
                            for (int j = 0; j < p1; ++j) {
                                const double lab = s.L1[q * p1 + i] * s.L1[q * p1 + j];
                                fp[i * p1 + j] += std::max(a, 0.0) * lab;
                                fn[i * p1 + j] += std::min(a, 0.0) * lab;
                            }
                    }
                }
    }

    // ---- parallel block Jacobi sweep (Sec. 6.5): tiles of the bounding box by
    //      the mean of each element's corner control points; inflow from another
    //      tile is lagged (previous sweep) and is no dependency ----
    s.tile.assign(ne, 0);
    if (in.sweep_tiles > 1) {
        const int T = in.sweep_tiles, m = in.m, nc = (m + 1) * (m + 1);
        double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
        for (size_t k = 0; k < (size_t)ne * nc; ++k)
            for (int c = 0; c < 2; ++c) {
                const double v = in.nodes[2 * (size_t)in.elem_nodes[k] + c];
                lo[c] = std::min(lo[c], v);
                hi[c] = std::max(hi[c], v);
            }
        const int cidx[4] = {0, m, m * (m + 1), m * (m + 1) + m};
        for (int e = 0; e < ne; ++e) {
            int t[2];
            for (int c = 0; c < 2; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 4; ++k) acc += in.nodes[2 * (size_t)in.elem_nodes[(size_t)e * nc + cidx[k]] + c];
                const double cen = acc / 4.0;
                t[c] = std::min((int)((cen - lo[c]) / (hi[c] - lo[c]) * T), T - 1);
            }
            s.tile[e] = t[1] * T + t[0];
        }
        for (int e = 0; e < ne; ++e)
            for (int f = 0; f < 4; ++f) {
                const int e2 = s.nbr[e * 4 + f];
                if (e2 < 0 || s.tile[e2] == s.tile[e]) continue;
                for (int d = 0; d < nd; ++d) {
                    int8_t& fd = s.fdir[((size_t)e * nd + d) * 4 + f];
                    if (fd == -1) fd = -2;
                    else if (fd == 2) fd = 3;
                }
            }
    }

    // ---- upwind levels per ordinate (Kahn), task list sorted by (level, e, d).
    //      An element depends on the neighbour across each face through which
    //      the ordinate enters it (fdir -1 or 2).  When no element is ready but
    //      some remain (a cycle), the lowest-numbered remaining element is taken
    //      next and its faces toward neighbours not yet done are lagged (fdir
    //      -1 -> -2, 2 -> 3: those values come from the previous sweep), the
    //      cycle lagging of Sec. 6.2 ----
    s.level.assign((size_t)nd * ne, -1);
    int maxlev = 0;
    int64_t lagged = 0;
    {
        auto pending = [&](int e, int d, int f) {  // face f of e is an unlagged inflow face from a neighbour
            const int8_t c = s.fdir[((size_t)e * nd + d) * 4 + f];
            return s.nbr[e * 4 + f] >= 0 && (c == -1 || c == 2);
        };
        std::vector<int> indeg(ne), queue(ne);
        std::vector<char> done(ne);
        for (int d = 0; d < nd; ++d) {
            int* lev = &s.level[(size_t)d * ne];
            int head = 0, tail = 0, low = 0;
            std::fill(done.begin(), done.end(), 0);
            for (int e = 0; e < ne; ++e) {
                int c = 0;
                for (int f = 0; f < 4; ++f) c += pending(e, d, f) ? 1 : 0;
                indeg[e] = c;
                if (c == 0) { lev[e] = 0; queue[tail++] = e; }
            }
            while (tail < ne || head < tail) {
                if (head == tail) {
                    if (!in.lag_cycles) { err = "an ordinate's upwind graph has a cycle"; return 5; }
                    while (done[low] || indeg[low] == 0) ++low;  // the lowest-numbered remaining element
                    const int v = low;
                    for (int f = 0; f < 4; ++f) {
                        const int u = s.nbr[v * 4 + f];
                        if (!pending(v, d, f) || done[u]) continue;
                        int8_t& c = s.fdir[((size_t)v * nd + d) * 4 + f];
                        c = c == -1 ? -2 : 3;
                        lagged += 1;
                    }
                    indeg[v] = 0;
                    lev[v] = std::max(lev[v], 0);
                    queue[tail++] = v;
                }
                const int u = queue[head++];
                done[u] = 1;
                for (int f = 0; f < 4; ++f) {
                    const int v = s.nbr[u * 4 + f];
                    if (v < 0 || !pending(v, d, s.nbr_face[u * 4 + f])) continue;  // v takes inflow from u
                    lev[v] = std::max(lev[v], lev[u] + 1);
                    if (--indeg[v] == 0) queue[tail++] = v;
                }
            }
            for (int e = 0; e < ne; ++e) maxlev = std::max(maxlev, lev[e]);
        }
    }
    s.n_cycle_lagged = lagged;
    s.nlevels = maxlev + 1;
    {
        std::vector<int64_t> cnt(s.nlevels + 1, 0);
        for (int d = 0; d < nd; ++d)
            for (int e = 0; e < ne; ++e) cnt[s.level[(size_t)d * ne + e] + 1]++;
        for (int l = 0; l < s.nlevels; ++l) cnt[l + 1] += cnt[l];
        s.level_start.assign(s.nlevels + 1, 0);
        for (int l = 0; l <= s.nlevels; ++l) s.level_start[l] = (int32_t)cnt[l];
        s.tasks.assign((size_t)ne * nd, 0);
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int e = 0; e < ne; ++e)
            for (int d = 0; d < nd; ++d) s.tasks[pos[s.level[(size_t)d * ne + e]]++] = e * nd + d;
    }

    // ---- sources and inflow, reorganized element-major ----
    if (in.source_kind == 0) {
        s.src.assign(in.q, in.q + (size_t)ne * n);
    } else {
        s.src.resize((size_t)ne * nd * n);
        for (int d = 0; d < nd; ++d)
            for (int e = 0; e < ne; ++e)
                for (int i = 0; i < n; ++i) s.src[((size_t)e * nd + d) * n + i] = in.q[((size_t)d * ne + e) * n + i];
    }
    s.inflow.clear();
    if (in.inflow_kind == 1 && s.nb > 0) {
        if (!in.inflow) { err = "nodal inflow requested without data"; return 1; }
        s.inflow.resize((size_t)s.nb * nd * p1);
        for (int d = 0; d < nd; ++d)
            for (int b = 0; b < s.nb; ++b)
                for (int a = 0; a < p1; ++a)
                    s.inflow[((size_t)b * nd + d) * p1 + a] = in.inflow[((size_t)d * s.nb + b) * p1 + a];
    }

    // ---- boundary data: unit normals, ds, E_b0 (Eq. eb0_disc) ----
    s.b_nhat.assign((size_t)s.nb * nfq * 2, 0.0);
    s.b_ds.assign((size_t)s.nb * nfq, 0.0);
    s.b_eb0.assign((size_t)s.nb * nfq, 0.0);
    for (int b = 0; b < s.nb; ++b) {
        int e = s.bface_elem[b], f = s.bface_face[b];
        for (int q = 0; q < nfq; ++q) {
            const double* nds = &s.nds[(((size_t)e * 4 + f) * nfq + q) * 2];
            double ds = std::sqrt(nds[0] * nds[0] + nds[1] * nds[1]);
            double nx = nds[0] / ds, ny = nds[1] / ds;
            s.b_nhat[((size_t)b * nfq + q) * 2] = nx;
            s.b_nhat[((size_t)b * nfq + q) * 2 + 1] = ny;
            s.b_ds[(size_t)b * nfq + q] = ds;
            double acc = 0.0;
            for (int d = 0; d < nd; ++d) acc += s.quad.w[d] * std::fabs(s.quad.ox[d] * nx + s.quad.oy[d] * ny);
            s.b_eb0[(size_t)b * nfq + q] = acc / (4.0 * kPi);
        }
    }

    // ---- IP-SMM operator blocks (Eq. ipsmm, left-hand side) ----
    s.Adiag.assign((size_t)ne * n * n, 0.0);
    s.Aoff.assign((size_t)ne * 4 * n * n, 0.0);
    s.Pinv.assign((size_t)ne * n * n, 0.0);
    if (in.moment_cg) s.Kcg.assign((size_t)ne * n * n, 0.0);
    int sing = 0;
#pragma omp parallel for schedule(static) reduction(+ : sing)
    for (int e = 0; e < ne; ++e) {
        const double st = s.sigma_t[e], sa = s.sigma_t[e] - s.sigma_s[e], D = 1.0 / (3.0 * st);
        double* Ad = &s.Adiag[(size_t)e * n * n];
        for (size_t ij = 0; ij < (size_t)n * n; ++ij)
            Ad[ij] = D * (s.Kxx[(size_t)e * n * n + ij] + s.Kyy[(size_t)e * n * n + ij]) + sa * s.M[(size_t)e * n * n + ij];
        std::vector<double> gn1(nfq * n), gn2(nfq * n);
        for (int f = 0; f < 4; ++f) {
            const size_t fo = ((size_t)e * 4 + f) * nfq;
            const double* V1 = &faceV[fo * n];
            const int e2 = s.nbr[e * 4 + f];
            if (e2 < 0) {
                int b = s.bface_id[e * 4 + f];
                for (int q = 0; q < nfq; ++q) {
                    double c = s.b_eb0[(size_t)b * nfq + q] * s.b_ds[(size_t)b * nfq + q];
                    for (int i = 0; i < n; ++i)
                        for (int j = 0; j < n; ++j) Ad[(size_t)i * n + j] += c * V1[q * n + i] * V1[q * n + j];
                }
                continue;
            }

            const int f2 = s.nbr_face[e * 4 + f], flip = s.nbr_flip[e * 4 + f];
            const double st2 = s.sigma_t[e2], D2 = 1.0 / (3.0 * st2);
            const double kappa = in.kappa_scale * 0.5 *
                                 (p1 * p1 / (st * s.hK[e]) + p1 * p1 / (st2 * s.hK[e2]));
            double* Ao = &s.Aoff[((size_t)e * 4 + f) * n * n];
            for (int q = 0; q < nfq; ++q) {
                const int q2 = flip ? nfq - 1 - q : q;
                const size_t fo2 = ((size_t)e2 * 4 + f2) * nfq + q2;
                const double* nds = &s.nds[(fo + q) * 2];
                for (int j = 0; j < n; ++j) {
                    gn1[q * n + j] = 0.5 * D * (s.Dfx[(fo + q) * n + j] * nds[0] + s.Dfy[(fo + q) * n + j] * nds[1]);
                    gn2[q * n + j] = 0.5 * D2 * (s.Dfx[fo2 * n + j] * nds[0] + s.Dfy[fo2 * n + j] * nds[1]);
                }
            }
            for (int q = 0; q < nfq; ++q) {
                const int q2 = flip ? nfq - 1 - q : q;
                const double* V2 = &faceV[(((size_t)e2 * 4 + f2) * nfq + q2) * n];
                const double* nds = &s.nds[(fo + q) * 2];
                const double ds = std::sqrt(nds[0] * nds[0] + nds[1] * nds[1]);
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) {
                        // self: kappa V1 V1 - V1 Gn1 - Gn1 V1
                        Ad[(size_t)i * n + j] += kappa * ds * V1[q * n + i] * V1[q * n + j]
                                                 - V1[q * n + i] * gn1[q * n + j] - gn1[q * n + i] * V1[q * n + j];
                        // coupling to the neighbour: -kappa V1 V2 - V1 Gn2 + Gn1 V2
                        Ao[(size_t)i * n + j] += -kappa * ds * V1[q * n + i] * V2[j]
                                                 - V1[q * n + i] * gn2[q * n + j] + gn1[q * n + i] * V2[j];
                    }
            }
        }
        if (!invert(n, Ad, &s.Pinv[(size_t)e * n * n])) sing += 1;
    }
    if (sing) { err = "singular diagonal block of the moment operator"; return 4; }
    if (int rc = factor_face_blocks(s, err)) return rc;

    // ---- continuous (CG) moment system (Sec. 5.1): element blocks without any
    //      interior-face term, and the continuous node numbering ----
    if (in.moment_cg) {
#pragma omp parallel for schedule(static)
        for (int e = 0; e < ne; ++e) {
            const double sa = s.sigma_t[e] - s.sigma_s[e], D = 1.0 / (3.0 * s.sigma_t[e]);
            double* Kc = &s.Kcg[(size_t)e * n * n];
            for (size_t ij = 0; ij < (size_t)n * n; ++ij)
                Kc[ij] = D * (s.Kxx[(size_t)e * n * n + ij] + s.Kyy[(size_t)e * n * n + ij]) + sa * s.M[(size_t)e * n * n + ij];
            for (int f = 0; f < 4; ++f) {
                if (s.nbr[e * 4 + f] >= 0) continue;
                const int b = s.bface_id[e * 4 + f];
                const double* V1 = &faceV[((size_t)e * 4 + f) * nfq * n];
                for (int q = 0; q < nfq; ++q) {
                    const double c = s.b_eb0[(size_t)b * nfq + q] * s.b_ds[(size_t)b * nfq + q];
                    for (int i = 0; i < n; ++i)
                        for (int j = 0; j < n; ++j) Kc[(size_t)i * n + j] += c * V1[q * n + i] * V1[q * n + j];
                }
            }
        }
        continuous_numbering(s);
    }

    // ---- fixed right-hand side: Q_0, Q_1 and J_in terms of Eq. ipsmm ----
    // Q_0 = sum_d w_d q_d, Q_1 = sum_d w_d Omega_d q_d (nodal)
    std::vector<double> Q((size_t)3 * ne * n, 0.0);
    for (int e = 0; e < ne; ++e)
        for (int d = 0; d < nd; ++d) {
            const double* qd = in.source_kind == 0 ? &s.src[(size_t)e * n] : &s.src[((size_t)e * nd + d) * n];
            for (int i = 0; i < n; ++i) {
                Q[(size_t)e * n + i] += s.quad.w[d] * qd[i];
                Q[((size_t)ne + e) * n + i] += s.quad.w[d] * s.quad.ox[d] * qd[i];
                Q[((size_t)2 * ne + e) * n + i] += s.quad.w[d] * s.quad.oy[d] * qd[i];
            }
        }
    s.bfixed.assign((size_t)ne * n, 0.0);
#pragma omp parallel for schedule(static)
    for (int e = 0; e < ne; ++e) {
        const double st = s.sigma_t[e];
        double* b = &s.bfixed[(size_t)e * n];
        const double* M = &s.M[(size_t)e * n * n];
        const double* Gx = &s.Gx[(size_t)e * n * n];
        const double* Gy = &s.Gy[(size_t)e * n * n];
        const double* q0 = &Q[(size_t)e * n];
        const double* q1x = &Q[((size_t)ne + e) * n];
        const double* q1y = &Q[((size_t)2 * ne + e) * n];
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j)
                acc += M[(size_t)i * n + j] * q0[j] + (Gx[(size_t)i * n + j] * q1x[j] + Gy[(size_t)i * n + j] * q1y[j]) / st;
            b[i] = acc;
        }
        for (int f = 0; f < 4; ++f) {
            const size_t fo = ((size_t)e * 4 + f) * nfq;
            const int e2 = s.nbr[e * 4 + f];
            if (e2 >= 0) {
                // - int_F u {Q_1 . n / sigma_t}
                const int f2 = s.nbr_face[e * 4 + f], flip = s.nbr_flip[e * 4 + f];
                const double st2 = s.sigma_t[e2];
                for (int q = 0; q < nfq; ++q) {
                    const int q2 = flip ? nfq - 1 - q : q;
                    const double* V1 = &faceV[(fo + q) * n];
                    const double* V2 = &faceV[(((size_t)e2 * 4 + f2) * nfq + q2) * n];
                    double a1x = 0, a1y = 0, a2x = 0, a2y = 0;
                    for (int j = 0; j < n; ++j) {
                        a1x += V1[j] * q1x[j];
                        a1y += V1[j] * q1y[j];
                        a2x += V2[j] * Q[((size_t)ne + e2) * n + j];
                        a2y += V2[j] * Q[((size_t)2 * ne + e2) * n + j];
                    }
                    const double* nds = &s.nds[(fo + q) * 2];
                    double g = 0.5 * ((a1x / st + a2x / st2) * nds[0] + (a1y / st + a2y / st2) * nds[1]);
                    for (int i = 0; i < n; ++i) b[i] -= V1[i] * g;
                }
            } else if (!s.inflow.empty()) {
                // - 2 int_F u J_in,  J_in = sum_{Omega.n<0} w (Omega.n) psibar
                const int bi = s.bface_id[e * 4 + f];
                for (int q = 0; q < nfq; ++q) {
                    const double nx = s.b_nhat[((size_t)bi * nfq + q) * 2], ny = s.b_nhat[((size_t)bi * nfq + q) * 2 + 1];
                    double jin = 0.0;
                    for (int d = 0; d < nd; ++d) {
                        double on = s.quad.ox[d] * nx + s.quad.oy[d] * ny;
                        if (!(on < 0.0)) continue;
                        double pb = 0.0;
                        for (int a = 0; a < p1; ++a) pb += s.L1[q * p1 + a] * s.inflow[((size_t)bi * nd + d) * p1 + a];
                        jin += s.quad.w[d] * on * pb;
                    }
                    const double* V1 = &faceV[(fo + q) * n];
                    const double c = 2.0 * jin * s.b_ds[(size_t)bi * nfq + q];
                    for (int i = 0; i < n; ++i) b[i] -= V1[i] * c;
                }
            }
        }
    }
    // T-source volume matrices scaled by -1/sigma_t
    for (int e = 0; e < ne; ++e) {
        const double c = -1.0 / s.sigma_t[e];
        for (size_t ij = 0; ij < (size_t)n * n; ++ij) {
            s.Kxx[(size_t)e * n * n + ij] *= c;
            s.Ks[(size_t)e * n * n + ij] *= c;
            s.Kyy[(size_t)e * n * n + ij] *= c;
        }
    }
    return 0;
}

}  // namespace smm
