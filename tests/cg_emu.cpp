// Test driver (CPU): the flexible-CG operator product of moments.cu
// (cgx_spmv_kernel: q = A p on the face-factored IP-SMM operator in FP32-pair
// arithmetic, two elements' rows per thread, and p.q through the last-block
// reduction) run on the host through host_kernel_shim.h, on the operator the
// library's host setup builds, stored as the library stores it (diagonal
// blocks and face couplings transposed, as FP32 pairs) and launched in the
// shape the library uses.  The kernel source and the helpers of blockops.cuh
// arrive as cg_kernels.inc, extracted by the test; the L2 cache-policy loads
// there are plain loads here.
// Usage: cg_emu DIR NE NNODES M P
//   in:  DIR/nodes.f64, elem.i32, sigma_t.f64, sigma_s.f64, q.f64 [ne][n], DIR/p.f64 [ne][n]
//   out: DIR/q_out.f64 [ne][n] (A p), DIR/scal.f64 [8] (scal[1] = p.q, scal[5] = scal[0] / p.q)
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "host_kernel_shim.h"
#include "setup.hpp"

namespace smm {
#include "cg_kernels.inc"
}

template <class T>
static bool read_file(const std::string& path, std::vector<T>& v) {
    std::ifstream in(path, std::ios::binary);
    in.read(reinterpret_cast<char*>(v.data()), (std::streamsize)(v.size() * sizeof(T)));
    return (bool)in;
}

template <class T>
static bool write_file(const std::string& path, const std::vector<T>& v) {
    std::ofstream out(path, std::ios::binary);
    out.write(reinterpret_cast<const char*>(v.data()), (std::streamsize)(v.size() * sizeof(T)));
    return (bool)out;
}

static std::vector<float2> pairs_of_transposed(const std::vector<double>& a, int n) {
    std::vector<float2> t(a.size());
    const size_t nb = a.size() / ((size_t)n * n);
    for (size_t b = 0; b < nb; ++b)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) t[b * n * n + (size_t)j * n + i] = smm::df_make(a[b * n * n + (size_t)i * n + j]);
    return t;
}

template <int N>
static void run(const smm::Setup& s, const std::vector<double>& p, std::vector<double>& q, std::vector<double>& scal) {
    const int ne = s.ne, n = s.n;
    const auto AdT2 = pairs_of_transposed(s.Adiag, n), CT2 = pairs_of_transposed(s.Cface, 2 * s.p1);
    std::vector<float2> p2(p.size());
    for (size_t i = 0; i < p.size(); ++i) p2[i] = smm::df_make(p[i]);
    const int tpb = std::max(1, 256 / n) * n, epb = tpb / n;
    constexpr int R = 2;
    const int nblk = (ne + epb * R - 1) / (epb * R);
    std::vector<double> part(nblk);
    std::vector<int> ctl(8, 0);
    scal.assign(8, 0.0);
    scal[0] = 1.0;
    q.assign((size_t)ne * n, 0.0);
    smm::CGArgs a{};
    a.ne = ne; a.n = n; a.nrow = ne * n;
    a.A2.AdT = AdT2.data(); a.A2.CT = CT2.data(); a.A2.nbr = s.nbr.data(); a.A2.nface = s.nbr_face.data();
    for (int k = 0; k < s.p1; ++k) a.A2.wd[k] = smm::df_make(s.wd[k]);
    a.p2 = p2.data(); a.p = const_cast<double*>(p.data()); a.q = q.data(); a.part = part.data();
    a.scal = scal.data(); a.ctl = ctl.data();
    emu_launch(nblk, tpb, 0, [&] { smm::cgx_spmv_kernel<N, R>(a); });
}

int main(int argc, char** argv) {
    if (argc != 6) return 2;
    const std::string dir = argv[1];
    const int ne = std::atoi(argv[2]), nn = std::atoi(argv[3]), m = std::atoi(argv[4]), p = std::atoi(argv[5]);
    const int n = (p + 1) * (p + 1);
    std::vector<double> nodes((size_t)nn * 2), st(ne), ss(ne), qs((size_t)ne * n), pv((size_t)ne * n);
    std::vector<int32_t> elem((size_t)ne * (m + 1) * (m + 1));
    if (!read_file(dir + "/nodes.f64", nodes) || !read_file(dir + "/elem.i32", elem) ||
        !read_file(dir + "/sigma_t.f64", st) || !read_file(dir + "/sigma_s.f64", ss) ||
        !read_file(dir + "/q.f64", qs) || !read_file(dir + "/p.f64", pv))
        return 3;
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
    std::vector<double> q, scal;
    switch (n) {
        case 4: run<4>(s, pv, q, scal); break;
        case 9: run<9>(s, pv, q, scal); break;
        case 16: run<16>(s, pv, q, scal); break;
        default: run<25>(s, pv, q, scal); break;
    }
    return write_file(dir + "/q_out.f64", q) && write_file(dir + "/scal.f64", scal) ? 0 : 5;
}
