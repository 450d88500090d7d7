// Host construction of the moment-system multigrid hierarchy (see amg.hpp).
#include "amg.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace smm {

namespace {

void spmv(const CSR& A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A.nrow; ++i) {
        double s = 0.0;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.v[k] * x[A.ci[k]];
        y[i] = s;
    }
}

CSR transpose(const CSR& A) {
    CSR T;
    T.nrow = A.ncol;
    T.ncol = A.nrow;
    T.rp.assign(T.nrow + 1, 0);
    for (int c : A.ci) T.rp[c + 1]++;
    for (int i = 0; i < T.nrow; ++i) T.rp[i + 1] += T.rp[i];
    T.ci.resize(A.ci.size());
    T.v.resize(A.v.size());
    std::vector<int> pos(T.rp.begin(), T.rp.end() - 1);
    for (int i = 0; i < A.nrow; ++i)
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            int p = pos[A.ci[k]]++;
            T.ci[p] = i;
            T.v[p] = A.v[k];
        }
    return T;
}

// C = A * B (Gustavson, columns sorted per row)
CSR multiply(const CSR& A, const CSR& B) {
    CSR C;
    C.nrow = A.nrow;
    C.ncol = B.ncol;
    C.rp.assign(C.nrow + 1, 0);
    std::vector<double> acc(B.ncol, 0.0);
    std::vector<int> mark(B.ncol, -1), cols;
    for (int i = 0; i < A.nrow; ++i) {
        cols.clear();
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            const int r = A.ci[k];
            const double a = A.v[k];
            for (int t = B.rp[r]; t < B.rp[r + 1]; ++t) {
                const int c = B.ci[t];
                if (mark[c] != i) {
                    mark[c] = i;
                    acc[c] = 0.0;
                    cols.push_back(c);
                }
                acc[c] += a * B.v[t];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int c : cols) {
            C.ci.push_back(c);
            C.v.push_back(acc[c]);
        }
        C.rp[i + 1] = (int)C.ci.size();
    }
    return C;
}

std::vector<double> diag_inv(const CSR& A) {
    std::vector<double> d(A.nrow, 0.0);
    for (int i = 0; i < A.nrow; ++i)
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (A.ci[k] == i) d[i] = 1.0 / A.v[k];
    return d;
}

// largest eigenvalue of D^{-1} A (A SPD) by power iteration with the
// Rayleigh quotient x^T A x / x^T D x
double lambda_max_jacobi(const CSR& A, const std::vector<double>& dinv, int iters = 30) {
    const int n = A.nrow;
    std::vector<double> x(n), y(n);
    for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.5 * std::sin(0.7 * i + 0.3);
    double lam = 1.0;
    for (int it = 0; it < iters; ++it) {
        spmv(A, x.data(), y.data());
        double xay = 0.0, xdx = 0.0;
        for (int i = 0; i < n; ++i) { xay += x[i] * y[i]; xdx += x[i] * x[i] / dinv[i]; }
        lam = xay / xdx;
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) { y[i] *= dinv[i]; nrm += y[i] * y[i]; }
        nrm = std::sqrt(nrm);
        for (int i = 0; i < n; ++i) x[i] = y[i] / nrm;
    }
    return lam;
}

// strength-based aggregation (three passes); returns aggregate id per node
std::vector<int> aggregate(const CSR& A, double theta, int& nagg) {
    const int n = A.nrow;
    std::vector<double> d(n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (A.ci[k] == i) d[i] = std::fabs(A.v[k]);
    auto strong = [&](int i, int k) {
        const int j = A.ci[k];
        return j != i && std::fabs(A.v[k]) >= theta * std::sqrt(d[i] * d[j]);
    };
    std::vector<int> agg(n, -1);
    nagg = 0;
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        bool free_nbhd = true;
        for (int k = A.rp[i]; k < A.rp[i + 1] && free_nbhd; ++k)
            if (strong(i, k) && agg[A.ci[k]] >= 0) free_nbhd = false;
        if (!free_nbhd) continue;
        agg[i] = nagg;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (strong(i, k)) agg[A.ci[k]] = nagg;
        ++nagg;
    }
    const std::vector<int> first = agg;
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        double best = -1.0;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (strong(i, k) && first[A.ci[k]] >= 0 && std::fabs(A.v[k]) > best) {
                best = std::fabs(A.v[k]);
                agg[i] = first[A.ci[k]];
            }
    }
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        agg[i] = nagg;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (strong(i, k) && agg[A.ci[k]] < 0) agg[A.ci[k]] = nagg;
        ++nagg;
    }
    return agg;
}

// P = (I - omega D^{-1} A) P_tent with P_tent[i][agg[i]] = 1
CSR smoothed_prolongator(const CSR& A, const std::vector<int>& agg, int nagg, double omega) {
    CSR P;
    P.nrow = A.nrow;
    P.ncol = nagg;
    P.rp.assign(A.nrow + 1, 0);
    std::vector<double> acc(nagg, 0.0);
    std::vector<int> mark(nagg, -1), cols;
    for (int i = 0; i < A.nrow; ++i) {
        double aii = 0.0;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (A.ci[k] == i) aii = A.v[k];
        cols.clear();
        auto add = [&](int c, double v) {
            if (mark[c] != i) { mark[c] = i; acc[c] = 0.0; cols.push_back(c); }
            acc[c] += v;
        };
        add(agg[i], 1.0);
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) add(agg[A.ci[k]], -omega * A.v[k] / aii);
        std::sort(cols.begin(), cols.end());
        for (int c : cols)
            if (acc[c] != 0.0) { P.ci.push_back(c); P.v.push_back(acc[c]); }
        P.rp[i + 1] = (int)P.ci.size();
    }
    return P;
}

bool dense_inverse(int n, const std::vector<double>& A, std::vector<double>& Ainv) {
    std::vector<double> a(A), b((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) b[(size_t)i * n + i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(a[(size_t)i * n + k]) > std::fabs(a[(size_t)piv * n + k])) piv = i;
        if (a[(size_t)piv * n + k] == 0.0) return false;
        if (piv != k)
            for (int j = 0; j < n; ++j) {
                std::swap(a[(size_t)k * n + j], a[(size_t)piv * n + j]);
                std::swap(b[(size_t)k * n + j], b[(size_t)piv * n + j]);
            }
        const double inv = 1.0 / a[(size_t)k * n + k];
        for (int j = 0; j < n; ++j) { a[(size_t)k * n + j] *= inv; b[(size_t)k * n + j] *= inv; }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            const double l = a[(size_t)i * n + k];
            if (l == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
                b[(size_t)i * n + j] -= l * b[(size_t)k * n + j];
            }
        }
    }
    Ainv.swap(b);
    return true;
}

}  // namespace

bool build_multigrid(int ne, int n, const std::vector<double>& Adiag, const std::vector<double>& Aoff,
                     const std::vector<double>& Pinv, const std::vector<int>& nbr, const std::vector<int>& corner_ids,
                     const std::vector<double>& gll, MGHierarchy& mg, std::string& err, int coarse_max) {
    mg = MGHierarchy();
    const size_t nn = (size_t)n * n;
    // ---- level-0 block-Jacobi damping: lambda_max(Pinv A) by power iteration
    //      (skipped when no block inverses are given: a continuous-space
    //      operator, whose level 0 the caller smooths itself) ----
    if (!Pinv.empty()) {
        const size_t N = (size_t)ne * n;
        std::vector<double> x(N), y(N), z(N);
        for (size_t i = 0; i < N; ++i) x[i] = 1.0 + 0.5 * std::sin(0.7 * (double)i + 0.3);
        double lam = 1.0;
        for (int it = 0; it < 30; ++it) {
#pragma omp parallel for schedule(static)
            for (int e = 0; e < ne; ++e) {
                for (int i = 0; i < n; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < n; ++j) s += Adiag[e * nn + (size_t)i * n + j] * x[(size_t)e * n + j];
                    for (int f = 0; f < 4; ++f) {
                        const int e2 = nbr[e * 4 + f];
                        if (e2 < 0) continue;
                        const double* B = &Aoff[((size_t)e * 4 + f) * nn];
                        for (int j = 0; j < n; ++j) s += B[(size_t)i * n + j] * x[(size_t)e2 * n + j];
                    }
                    y[(size_t)e * n + i] = s;
                }
                for (int i = 0; i < n; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < n; ++j) s += Pinv[e * nn + (size_t)i * n + j] * y[(size_t)e * n + j];
                    z[(size_t)e * n + i] = s;
                }
            }
            // Rayleigh quotient x^T A x / x^T Adiag x
            double xay = 0.0, xdx = 0.0, nrm = 0.0;
            for (int e = 0; e < ne; ++e)
                for (int i = 0; i < n; ++i) {
                    double dx = 0.0;
                    for (int j = 0; j < n; ++j) dx += Adiag[e * nn + (size_t)i * n + j] * x[(size_t)e * n + j];
                    xay += x[(size_t)e * n + i] * y[(size_t)e * n + i];
                    xdx += x[(size_t)e * n + i] * dx;
                }
            lam = xay / xdx;
            for (size_t i = 0; i < N; ++i) nrm += z[i] * z[i];
            nrm = std::sqrt(nrm);
            for (size_t i = 0; i < N; ++i) x[i] = z[i] / nrm;
        }
        mg.omega0 = (4.0 / 3.0) / (1.05 * lam);
    }
    // ---- level 1: continuous bilinear functions on the mesh vertices ----
    {
        std::vector<int> ids(corner_ids);
        std::vector<int> sorted(ids);
        std::sort(sorted.begin(), sorted.end());
        sorted.erase(std::unique(sorted.begin(), sorted.end()), sorted.end());
        mg.nvert = (int)sorted.size();
        mg.vid.resize(ids.size());
        for (size_t k = 0; k < ids.size(); ++k)
            mg.vid[k] = (int)(std::lower_bound(sorted.begin(), sorted.end(), ids[k]) - sorted.begin());
        const int p1 = (int)gll.size();
        mg.w4.assign((size_t)n * 4, 0.0);
        for (int iy = 0; iy < p1; ++iy)
            for (int ix = 0; ix < p1; ++ix) {
                const double x = gll[ix], y = gll[iy];
                double* w = &mg.w4[(size_t)(iy * p1 + ix) * 4];
                w[0] = (1 - x) * (1 - y);
                w[1] = x * (1 - y);
                w[2] = (1 - x) * y;
                w[3] = x * y;
            }
        mg.vrp.assign(mg.nvert + 1, 0);
        for (int v : mg.vid) mg.vrp[v + 1]++;
        for (int v = 0; v < mg.nvert; ++v) mg.vrp[v + 1] += mg.vrp[v];
        mg.vinc.assign(mg.vid.size(), 0);
        std::vector<int> pos(mg.vrp.begin(), mg.vrp.end() - 1);
        for (size_t k = 0; k < mg.vid.size(); ++k) mg.vinc[pos[mg.vid[k]]++] = (int)k;
    }
    MGLevel L1;
    {
        // 4x4 Galerkin block W^T B W for every operator block B
        auto galerkin4 = [&](const double* B, double out[16]) {
            double t[4 * 64];
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < 4; ++k) {
                    double s = 0.0;
                    for (int j = 0; j < n; ++j) s += B[(size_t)i * n + j] * mg.w4[(size_t)j * 4 + k];
                    t[i * 4 + k] = s;
                }
            for (int a = 0; a < 4; ++a)
                for (int k = 0; k < 4; ++k) {
                    double s = 0.0;
                    for (int i = 0; i < n; ++i) s += mg.w4[(size_t)i * 4 + a] * t[i * 4 + k];
                    out[a * 4 + k] = s;
                }
        };
        std::vector<std::vector<std::pair<int, double>>> rows(mg.nvert);
        for (int e = 0; e < ne; ++e) {
            double g[16];
            galerkin4(&Adiag[e * nn], g);
            for (int a = 0; a < 4; ++a)
                for (int k = 0; k < 4; ++k) rows[mg.vid[e * 4 + a]].push_back({mg.vid[e * 4 + k], g[a * 4 + k]});
            for (int f = 0; f < 4; ++f) {
                const int e2 = nbr[e * 4 + f];
                if (e2 < 0 || Aoff.empty()) continue;
                galerkin4(&Aoff[((size_t)e * 4 + f) * nn], g);
                for (int a = 0; a < 4; ++a)
                    for (int k = 0; k < 4; ++k) rows[mg.vid[e * 4 + a]].push_back({mg.vid[e2 * 4 + k], g[a * 4 + k]});
            }
        }
        L1.A.nrow = L1.A.ncol = mg.nvert;
        L1.A.rp.assign(mg.nvert + 1, 0);
        for (int v = 0; v < mg.nvert; ++v) {
            auto& r = rows[v];
            std::sort(r.begin(), r.end(), [](const std::pair<int, double>& a, const std::pair<int, double>& b) {
                return a.first < b.first;
            });
            for (size_t k = 0; k < r.size(); ++k) {
                if (k > 0 && r[k].first == r[k - 1].first) {
                    L1.A.v.back() += r[k].second;
                } else {
                    L1.A.ci.push_back(r[k].first);
                    L1.A.v.push_back(r[k].second);
                }
            }
            L1.A.rp[v + 1] = (int)L1.A.ci.size();
            std::vector<std::pair<int, double>>().swap(r);
        }
    }
    mg.lv.clear();
    mg.lv.emplace_back();  // level 0 placeholder
    mg.lv.push_back(std::move(L1));
    // ---- smoothed-aggregation levels ----
    while (mg.lv.back().A.nrow > coarse_max) {
        MGLevel& cur = mg.lv.back();
        cur.dinv = diag_inv(cur.A);
        const double lam = lambda_max_jacobi(cur.A, cur.dinv);
        int nagg = 0;
        std::vector<int> agg = aggregate(cur.A, 0.08, nagg);
        if (nagg >= cur.A.nrow || nagg == 0) break;
        cur.P = smoothed_prolongator(cur.A, agg, nagg, (4.0 / 3.0) / lam);
        cur.R = transpose(cur.P);
        MGLevel next;
        next.A = multiply(cur.R, multiply(cur.A, cur.P));
        const bool stalled = nagg > 0.8 * cur.A.nrow;
        mg.lv.push_back(std::move(next));
        if (stalled) break;
    }
    for (size_t l = 1; l < mg.lv.size(); ++l) {
        MGLevel& L = mg.lv[l];
        L.dinv = diag_inv(L.A);
        for (double d : L.dinv)
            if (!(d > 0.0) || !std::isfinite(d)) { err = "multigrid: non-positive diagonal"; return false; }
        L.omega = (4.0 / 3.0) / (1.05 * lambda_max_jacobi(L.A, L.dinv));
    }
    // ---- coarsest: dense inverse ----
    const CSR& C = mg.lv.back().A;
    mg.ncoarse = C.nrow;
    if (C.nrow > 4096) { err = "multigrid: coarsest level too large"; return false; }
    std::vector<double> dense((size_t)C.nrow * C.nrow, 0.0);
    for (int i = 0; i < C.nrow; ++i)
        for (int k = C.rp[i]; k < C.rp[i + 1]; ++k) dense[(size_t)i * C.nrow + C.ci[k]] += C.v[k];
    if (!dense_inverse(C.nrow, dense, mg.coarse_inv)) { err = "multigrid: singular coarsest operator"; return false; }
    return true;
}

}  // namespace smm
