// Test driver (CPU): one level-0 smoothing step of the moment-solve multigrid
// preconditioner (bj_smooth_kernel of mg.cu, FP32,
//   xout = xin + c2 Pinv (b - A xin) + c1 (xin - xprev)
// with A applied as its face couplings and Pinv = A_d^{-1}, two elements' rows
// per thread) run on the host through host_kernel_shim.h, on the FP32 copies of
// the face couplings and block inverses that the library's host setup builds,
// stored and launched as the library stores and launches them.  The kernel
// source and the helpers of blockops.cuh arrive as smooth_kernels.inc,
// extracted by the test.
// MODE 2 runs instead the last smoothing step of a V-cycle inside the flexible
// CG (bj_last_dots_kernel): the step in FP64 output z with b = r, the dots r.z
// and (r - r_old).z per block, and in the last block beta = (r - r_old).z /
// rz_old, the new rz, rr from the first step's partials, the iteration count
// and the convergence test.
// MODE 3 runs the first step of a V-cycle inside the flexible CG
// (bj_first_update_kernel): the CG update x += alpha p, r_old = r, r -= alpha q
// folded in, xout = c2 Pinv r, and the per-block partials of r.r.
//   MODE 3 in: DIR/b.f64 holds r, DIR/x.f64, p.f64, q.f64 [ne][n], DIR/cg.f64 (alpha);
//   out: DIR/x_out.f64, r_out.f64, rold_out.f64 [ne][n], DIR/xout.f32, DIR/rr.f64 (the partials)
// MODE 4 runs the level-0 residual restricted to the element corners
// (bj_residual_kernel): cres[e][c] = sum_i w4[i][c] (b - A x)[e][i] with the
// diagonal blocks entering as W = w4^T A_d, formed here as the library forms it.
//   MODE 4 in: DIR/b.f64 [ne][n], DIR/xin.f32 [ne][n], DIR/w4.f64 [n][4]; out: DIR/cres.f32 [ne][4]
// Usage: smooth_emu DIR NE NNODES M P C1 C2 MODE   (MODE 1: first step, 0: inner step, 2: last step)
//   in:  DIR/nodes.f64, elem.i32, sigma_t.f64, sigma_s.f64, q.f64 [ne][n], DIR/b.f64 [ne][n] (FP64; r in
//        MODE 2), DIR/xin.f32 and DIR/xprev.f32 [ne][n] (FP32; not read in MODE 1: xin = xprev = 0);
//        MODE 2 also DIR/rold.f64 [ne][n], DIR/cg.f64 (rz_old, rr threshold, then the first step's rr
//        partials, one per block)
//   out: DIR/xout.f32 [ne][n] (MODE 0, 1); MODE 2: DIR/z.f64 [ne][n], DIR/scal.f64 [8], DIR/ctl.i32 [8]
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "host_kernel_shim.h"
#include "setup.hpp"

namespace smm {
#include "smooth_kernels.inc"
}

template <class T>
static bool read_file(const std::string& path, std::vector<T>& v) {
    std::ifstream in(path, std::ios::binary);
    in.read(reinterpret_cast<char*>(v.data()), (std::streamsize)(v.size() * sizeof(T)));
    return (bool)in;
}

static std::vector<float> f32_transposed(const std::vector<double>& a, int n) {
    std::vector<float> t(a.size());
    const size_t nb = a.size() / ((size_t)n * n);
    for (size_t b = 0; b < nb; ++b)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) t[b * n * n + (size_t)j * n + i] = (float)a[b * n * n + (size_t)i * n + j];
    return t;
}

template <int N>
static void run(const smm::Setup& s, float c1, float c2, const std::vector<double>& b, const float* xin,
                const float* xprev, std::vector<float>& xout) {
    constexpr int R = 2;  // rows per thread, as the library launches the step
    const auto CT = f32_transposed(s.Cface, 2 * s.p1), PinvT = f32_transposed(s.Pinv, s.n);
    smm::FaceOp<float> A;
    A.CT = CT.data(); A.nbr = s.nbr.data(); A.nface = s.nbr_face.data();
    for (int k = 0; k < s.p1; ++k) A.wd[k] = (float)s.wd[k];
    const int tpb = std::max(1, 256 / N) * N, epb = smm::FaceDims<N>::EPB;
    const int nblk = (s.ne + epb * R - 1) / (epb * R);
    std::vector<int> ctl(8, 0);
    xout.assign((size_t)s.ne * N, 0.0f);
    emu_launch(nblk, tpb, 0, [&] {
        smm::bj_smooth_kernel<float, N, R>(s.ne, A, PinvT.data(), c1, c2, b.data(), xin, xprev, xout.data(),
                                           ctl.data());
    });
}

template <int N>
static bool run_last(const std::string& dir, const smm::Setup& s, float c1, float c2, std::vector<double>& r,
                     const std::vector<float>& xin, const std::vector<float>& xprev) {
    constexpr int R = 2;
    const int ne = s.ne;
    const auto CT = f32_transposed(s.Cface, 2 * s.p1), PinvT = f32_transposed(s.Pinv, s.n);
    smm::FaceOp<float> A;
    A.CT = CT.data(); A.nbr = s.nbr.data(); A.nface = s.nbr_face.data();
    for (int k = 0; k < s.p1; ++k) A.wd[k] = (float)s.wd[k];
    const int tpb = std::max(1, 256 / N) * N, epb = smm::FaceDims<N>::EPB;
    const int grid = (ne + epb * R - 1) / (epb * R);
    const int nblk = grid + 3;  // the row kernels' block count sets the partials' stride; any count >= grid
    std::vector<double> rold((size_t)ne * N), cg(2 + grid), z((size_t)ne * N, 0.0), part(4 * (size_t)nblk, 0.0);
    if (!read_file(dir + "/rold.f64", rold) || !read_file(dir + "/cg.f64", cg)) return false;
    for (int b = 0; b < grid; ++b) part[nblk + b] = cg[2 + b];
    std::vector<double> scal(8, 0.0);
    std::vector<int> ctl(8, 0);
    scal[0] = cg[0];
    scal[4] = cg[1];
    ctl[1] = 5;   // iterations so far
    ctl[2] = 100; // iteration limit
    smm::CGArgs a{};
    a.ne = ne; a.n = N; a.nrow = ne * N; a.nblk = nblk;
    a.r = r.data(); a.rold = rold.data(); a.z = z.data(); a.part = part.data(); a.scal = scal.data();
    a.ctl = ctl.data();
    emu_launch(grid, tpb, 0, [&] {
        smm::bj_last_dots_kernel<N, R>(a, A, PinvT.data(), c1, c2, xin.data(), xprev.data());
    });
    std::ofstream oz(dir + "/z.f64", std::ios::binary), os(dir + "/scal.f64", std::ios::binary),
        oc(dir + "/ctl.i32", std::ios::binary);
    oz.write(reinterpret_cast<const char*>(z.data()), (std::streamsize)(z.size() * sizeof(double)));
    os.write(reinterpret_cast<const char*>(scal.data()), (std::streamsize)(scal.size() * sizeof(double)));
    oc.write(reinterpret_cast<const char*>(ctl.data()), (std::streamsize)(ctl.size() * sizeof(int)));
    return (bool)oz && (bool)os && (bool)oc;
}

template <class T>
static bool write_vec(const std::string& path, const std::vector<T>& v) {
    std::ofstream out(path, std::ios::binary);
    out.write(reinterpret_cast<const char*>(v.data()), (std::streamsize)(v.size() * sizeof(T)));
    return (bool)out;
}

template <int N>
static bool run_first_update(const std::string& dir, const smm::Setup& s, float c2, std::vector<double>& r) {
    constexpr int R = 2;
    const int ne = s.ne;
    const auto PinvT = f32_transposed(s.Pinv, s.n);
    const int tpb = std::max(1, 256 / N) * N, epb = smm::FaceDims<N>::EPB;
    const int grid = (ne + epb * R - 1) / (epb * R);
    const int nblk = grid + 3;
    std::vector<double> x((size_t)ne * N), pv((size_t)ne * N), q((size_t)ne * N), alpha(1);
    std::vector<double> rold((size_t)ne * N, 0.0), part(4 * (size_t)nblk, 0.0), scal(8, 0.0);
    std::vector<float> xout((size_t)ne * N, 0.0f);
    std::vector<int> ctl(8, 0);
    if (!read_file(dir + "/x.f64", x) || !read_file(dir + "/p.f64", pv) || !read_file(dir + "/q.f64", q) ||
        !read_file(dir + "/cg.f64", alpha))
        return false;
    scal[5] = alpha[0];
    smm::CGArgs a{};
    a.ne = ne; a.n = N; a.nrow = ne * N; a.nblk = nblk;
    a.x = x.data(); a.p = pv.data(); a.q = q.data(); a.r = r.data(); a.rold = rold.data(); a.part = part.data();
    a.scal = scal.data(); a.ctl = ctl.data();
    emu_launch(grid, tpb, 0, [&] { smm::bj_first_update_kernel<N, R>(a, PinvT.data(), c2, xout.data()); });
    const std::vector<double> rr(part.begin() + nblk, part.begin() + nblk + grid);
    return write_vec(dir + "/x_out.f64", x) && write_vec(dir + "/r_out.f64", r) &&
           write_vec(dir + "/rold_out.f64", rold) && write_vec(dir + "/xout.f32", xout) && write_vec(dir + "/rr.f64", rr);
}

template <int N>
static bool run_residual(const std::string& dir, const smm::Setup& s, const std::vector<double>& b,
                         const std::vector<float>& x) {
    constexpr int R = 2;
    const int ne = s.ne;
    std::vector<double> w4d((size_t)N * 4);
    if (!read_file(dir + "/w4.f64", w4d)) return false;
    const std::vector<float> w4(w4d.begin(), w4d.end());
    std::vector<float> WdT((size_t)ne * N * 4);
    for (int e = 0; e < ne; ++e)
        for (int j = 0; j < N; ++j)
            for (int c = 0; c < 4; ++c) {
                double acc = 0.0;
                for (int i = 0; i < N; ++i) acc += w4d[(size_t)i * 4 + c] * s.Adiag[((size_t)e * N + i) * N + j];
                WdT[((size_t)e * N + j) * 4 + c] = (float)acc;
            }
    const auto CT = f32_transposed(s.Cface, 2 * s.p1);
    smm::FaceOp<float> A;
    A.CT = CT.data(); A.nbr = s.nbr.data(); A.nface = s.nbr_face.data();
    for (int k = 0; k < s.p1; ++k) A.wd[k] = (float)s.wd[k];
    const int tpb = std::max(1, 256 / N) * N, epb = smm::FaceDims<N>::EPB;
    const int grid = (ne + epb * R - 1) / (epb * R);
    std::vector<float> cres((size_t)ne * 4, 0.0f);
    std::vector<int> ctl(8, 0);
    emu_launch(grid, tpb, 0, [&] {
        smm::bj_residual_kernel<N, R>(ne, A, WdT.data(), b.data(), x.data(), w4.data(), cres.data(), nullptr, 0,
                                      ctl.data());
    });
    std::ofstream out(dir + "/cres.f32", std::ios::binary);
    out.write(reinterpret_cast<const char*>(cres.data()), (std::streamsize)(cres.size() * sizeof(float)));
    return (bool)out;
}

int main(int argc, char** argv) {
    if (argc != 9) return 2;
    const std::string dir = argv[1];
    const int ne = std::atoi(argv[2]), nn = std::atoi(argv[3]), m = std::atoi(argv[4]), p = std::atoi(argv[5]);
    const float c1 = (float)std::atof(argv[6]), c2 = (float)std::atof(argv[7]);
    const int mode = std::atoi(argv[8]);
    const bool first = mode == 1;
    const int n = (p + 1) * (p + 1);
    std::vector<double> nodes((size_t)nn * 2), st(ne), ss(ne), qs((size_t)ne * n), b((size_t)ne * n);
    std::vector<int32_t> elem((size_t)ne * (m + 1) * (m + 1));
    std::vector<float> xin((size_t)ne * n, 0.0f), xprev((size_t)ne * n, 0.0f), xout;
    if (!read_file(dir + "/nodes.f64", nodes) || !read_file(dir + "/elem.i32", elem) ||
        !read_file(dir + "/sigma_t.f64", st) || !read_file(dir + "/sigma_s.f64", ss) ||
        !read_file(dir + "/q.f64", qs) || !read_file(dir + "/b.f64", b))
        return 3;
    if ((mode == 0 || mode == 2) && (!read_file(dir + "/xin.f32", xin) || !read_file(dir + "/xprev.f32", xprev)))
        return 3;
    if (mode == 4 && !read_file(dir + "/xin.f32", xin)) return 3;
    smm::Input in;
    in.ne = ne; in.m = m; in.p = p; in.sn = 4; in.n_nodes = nn;
    in.nodes = nodes.data(); in.elem_nodes = elem.data(); in.sigma_t = st.data(); in.sigma_s = ss.data();
    in.q = qs.data();
    smm::Setup s;
    std::string err;
    if (smm::build_setup(in, s, err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    if (mode == 4) {
        bool ok = false;
        switch (n) {
            case 4: ok = run_residual<4>(dir, s, b, xin); break;
            case 9: ok = run_residual<9>(dir, s, b, xin); break;
            case 16: ok = run_residual<16>(dir, s, b, xin); break;
            default: ok = run_residual<25>(dir, s, b, xin); break;
        }
        return ok ? 0 : 5;
    }
    if (mode == 3) {
        bool ok = false;
        switch (n) {
            case 4: ok = run_first_update<4>(dir, s, c2, b); break;
            case 9: ok = run_first_update<9>(dir, s, c2, b); break;
            case 16: ok = run_first_update<16>(dir, s, c2, b); break;
            default: ok = run_first_update<25>(dir, s, c2, b); break;
        }
        return ok ? 0 : 5;
    }
    if (mode == 2) {
        bool ok = false;
        switch (n) {
            case 4: ok = run_last<4>(dir, s, c1, c2, b, xin, xprev); break;
            case 9: ok = run_last<9>(dir, s, c1, c2, b, xin, xprev); break;
            case 16: ok = run_last<16>(dir, s, c1, c2, b, xin, xprev); break;
            default: ok = run_last<25>(dir, s, c1, c2, b, xin, xprev); break;
        }
        return ok ? 0 : 5;
    }
    const float* xi = first ? nullptr : xin.data();
    const float* xp = first ? nullptr : xprev.data();
    switch (n) {
        case 4: run<4>(s, c1, c2, b, xi, xp, xout); break;
        case 9: run<9>(s, c1, c2, b, xi, xp, xout); break;
        case 16: run<16>(s, c1, c2, b, xi, xp, xout); break;
        default: run<25>(s, c1, c2, b, xi, xp, xout); break;
    }
    std::ofstream out(dir + "/xout.f32", std::ios::binary);
    out.write(reinterpret_cast<const char*>(xout.data()), (std::streamsize)(xout.size() * sizeof(float)));
    return out ? 0 : 5;
}
