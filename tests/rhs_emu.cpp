// Test driver (CPU): the IP-SMM right-hand-side kernels of moments.cu run on
// the host through host_kernel_shim.h, on the operators the library's host
// setup builds, uploaded in the library's layouts (K blocks column-major,
// face gradient operators point-major and node-major, all as FP32 pairs) and
// launched in the shapes of launch_rhs_n.  The kernel source arrives as
// rhs_kernels.inc, extracted from moments.cu by the test.
// Usage: rhs_emu DIR NE NNODES M P
//   in:  DIR/nodes.f64, elem.i32, sigma_t.f64, q.f64 (as setup_dump), DIR/mom.f64 [6][ne][n],
//        DIR/beta.f64 [n_bface][nfq]
//   out: DIR/dims.txt (n nfq n_bface), DIR/rhs.f64 [ne][n]
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "host_kernel_shim.h"
#include "setup.hpp"

namespace smm {
#include "rhs_kernels.inc"
}

template <class T>
static bool read_file(const std::string& path, std::vector<T>& v) {
    std::ifstream in(path, std::ios::binary);
    in.read(reinterpret_cast<char*>(v.data()), (std::streamsize)(v.size() * sizeof(T)));
    return (bool)in;
}

static std::vector<float2> pairs(const std::vector<double>& v) {
    std::vector<float2> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float hi = (float)v[i];
        out[i] = make_float2(hi, (float)(v[i] - (double)hi));
    }
    return out;
}

template <int N>
static void run(const smm::Setup& s, const std::vector<double>& mom, const std::vector<double>& beta,
                std::vector<double>& rhs) {
    const int ne = s.ne, n = s.n, nfq = s.nfq, p = s.p;
    std::vector<double> KxxT(s.Kxx.size()), KsT(s.Ks.size()), KyyT(s.Kyy.size());
    for (int e = 0; e < ne; ++e)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const size_t a = ((size_t)e * n + i) * n + j, b = ((size_t)e * n + j) * n + i;
                KxxT[b] = s.Kxx[a];
                KsT[b] = s.Ks[a];
                KyyT[b] = s.Kyy[a];
            }
    std::vector<double> tx(s.Dfx.size()), ty(s.Dfy.size());
    for (size_t b = 0; b < (size_t)ne * 4; ++b)
        for (int q = 0; q < nfq; ++q)
            for (int j = 0; j < n; ++j) {
                tx[(b * n + j) * nfq + q] = s.Dfx[(b * nfq + q) * n + j];
                ty[(b * n + j) * nfq + q] = s.Dfy[(b * nfq + q) * n + j];
            }
    const auto Kxx = pairs(KxxT), Ks = pairs(KsT), Kyy = pairs(KyyT);
    const auto Dfx = pairs(s.Dfx), Dfy = pairs(s.Dfy), DfxT = pairs(tx), DfyT = pairs(ty);
    std::vector<double> trace((size_t)ne * 4 * nfq * 3);
    rhs.assign((size_t)ne * n, 0.0);
    // the shapes of launch_rhs_n
    const int fq = 4 * nfq, ept = std::max(1, 256 / fq);
    emu_launch((ne + ept - 1) / ept, (ept * fq + 31) / 32 * 32, (size_t)3 * ept * n * sizeof(float2), [&] {
        smm::rhs_trace_kernel<N>(ne, n, p, nfq, ept, mom.data(), DfxT.data(), DfyT.data(), s.nds.data(), s.L1.data(),
                                 s.sigma_t.data(), trace.data());
    });
    const int epa = std::max(1, std::min(256 / n, 32));
    const size_t sh2 = (size_t)(3 * epa * n + 2 * epa * fq) * sizeof(float2) + (size_t)epa * fq * sizeof(double);
    emu_launch((ne + epa - 1) / epa, (epa * n + 31) / 32 * 32, sh2, [&] {
        smm::rhs_assemble_kernel<N>(ne, n, p, nfq, epa, mom.data(), beta.data(), s.bfixed.data(), Kxx.data(),
                                    Ks.data(), Kyy.data(), Dfx.data(), Dfy.data(), s.L1.data(), s.sigma_t.data(),
                                    s.nbr.data(), s.nbr_face.data(), s.nbr_flip.data(), s.bface_id.data(),
                                    s.b_ds.data(), trace.data(), rhs.data());
    });
}

int main(int argc, char** argv) {
    if (argc != 6) return 2;
    const std::string dir = argv[1];
    const int ne = std::atoi(argv[2]), nn = std::atoi(argv[3]), m = std::atoi(argv[4]), p = std::atoi(argv[5]);
    const int n = (p + 1) * (p + 1);
    std::vector<double> nodes((size_t)nn * 2), st(ne), ss(ne), q((size_t)ne * n);
    std::vector<int32_t> elem((size_t)ne * (m + 1) * (m + 1));
    if (!read_file(dir + "/nodes.f64", nodes) || !read_file(dir + "/elem.i32", elem) ||
        !read_file(dir + "/sigma_t.f64", st) || !read_file(dir + "/q.f64", q))
        return 3;
    for (int e = 0; e < ne; ++e) ss[e] = 0.5 * st[e];
    smm::Input in;
    in.ne = ne; in.m = m; in.p = p; in.sn = 4; in.n_nodes = nn;
    in.nodes = nodes.data(); in.elem_nodes = elem.data(); in.sigma_t = st.data(); in.sigma_s = ss.data();
    in.q = q.data();
    smm::Setup s;
    std::string err;
    if (smm::build_setup(in, s, err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    std::vector<double> mom((size_t)6 * ne * n), beta((size_t)s.nb * s.nfq), rhs;
    if (!read_file(dir + "/mom.f64", mom) || !read_file(dir + "/beta.f64", beta)) return 3;
    switch (n) {
        case 4: run<4>(s, mom, beta, rhs); break;
        case 9: run<9>(s, mom, beta, rhs); break;
        case 16: run<16>(s, mom, beta, rhs); break;
        case 25: run<25>(s, mom, beta, rhs); break;
        default: run<0>(s, mom, beta, rhs); break;
    }
    std::ofstream dims(dir + "/dims.txt");
    dims << s.n << " " << s.nfq << " " << s.nb << "\n";
    std::ofstream out(dir + "/rhs.f64", std::ios::binary);
    out.write(reinterpret_cast<const char*>(rhs.data()), (std::streamsize)(rhs.size() * sizeof(double)));
    return out && dims ? 0 : 5;
}
