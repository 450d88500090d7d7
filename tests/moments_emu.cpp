// Test driver (CPU): the angular-moment kernels of moments.cu (moments_kernel
// on FP64 psi, moments_df_kernel on its FP32-pair copy, beta_kernel at the
// boundary Gauss points) run on the host through host_kernel_shim.h, on the
// quadrature and boundary data the library's host setup builds, in the
// library's layouts and the launch shapes of launch_moments, launch_moments_df
// and launch_beta.  The kernel source arrives as moments_kernels.inc,
// extracted from moments.cu by the test.
// Usage: moments_emu DIR NE NNODES M P SN
//   in:  DIR/nodes.f64, elem.i32, sigma_t.f64, q.f64 (as setup_dump),
//        DIR/psi.f64 [ne][nd][n] (the device layout)
//   out: DIR/dims.txt (n nd nfq n_bface), DIR/mom.f64 and DIR/mom_df.f64 [6][ne][n],
//        DIR/beta.f64 [n_bface][nfq] (from the FP64 moments)
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "host_kernel_shim.h"
#include "setup.hpp"

namespace smm {
#include "moments_kernels.inc"
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

int main(int argc, char** argv) {
    if (argc != 7) return 2;
    const std::string dir = argv[1];
    const int ne = std::atoi(argv[2]), nn = std::atoi(argv[3]), m = std::atoi(argv[4]), p = std::atoi(argv[5]);
    const int sn = std::atoi(argv[6]);
    const int n = (p + 1) * (p + 1);
    std::vector<double> nodes((size_t)nn * 2), st(ne), ss(ne), q((size_t)ne * n);
    std::vector<int32_t> elem((size_t)ne * (m + 1) * (m + 1));
    if (!read_file(dir + "/nodes.f64", nodes) || !read_file(dir + "/elem.i32", elem) ||
        !read_file(dir + "/sigma_t.f64", st) || !read_file(dir + "/q.f64", q))
        return 3;
    for (int e = 0; e < ne; ++e) ss[e] = 0.5 * st[e];
    smm::Input in;
    in.ne = ne; in.m = m; in.p = p; in.sn = sn; in.n_nodes = nn;
    in.nodes = nodes.data(); in.elem_nodes = elem.data(); in.sigma_t = st.data(); in.sigma_s = ss.data();
    in.q = q.data();
    smm::Setup s;
    std::string err;
    if (smm::build_setup(in, s, err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    const int nd = s.nd, nfq = s.nfq, nb = s.nb;
    std::vector<double> psi((size_t)ne * nd * n);
    if (!read_file(dir + "/psi.f64", psi)) return 3;
    // the pair copy of psi and the six pair weights w_d (1, Ox, Oy, OxOx, OxOy, OyOy), as the library forms them
    std::vector<float2> psi2(psi.size()), wq((size_t)6 * nd);
    for (size_t i = 0; i < psi.size(); ++i) psi2[i] = smm::df_make(psi[i]);
    for (int d = 0; d < nd; ++d) {
        const double w = s.quad.w[d], x = s.quad.ox[d], y = s.quad.oy[d];
        const double v[6] = {w, w * x, w * y, w * x * x, w * x * y, w * y * y};
        for (int k = 0; k < 6; ++k) wq[(size_t)k * nd + d] = smm::df_make(v[k]);
    }
    std::vector<double> mom((size_t)6 * ne * n, 0.0), mom_df((size_t)6 * ne * n, 0.0), beta((size_t)nb * nfq, 0.0);
    const int grid = std::max(1, std::min((ne + 7) / 8, 65535));
    emu_launch(grid, 256, 0, [&] {
        smm::moments_kernel(ne, nd, n, s.quad.w.data(), s.quad.ox.data(), s.quad.oy.data(), psi.data(), mom.data());
    });
    emu_launch(grid, 256, 0, [&] { smm::moments_df_kernel(ne, nd, n, wq.data(), psi2.data(), mom_df.data()); });
    if (nb * nfq > 0)
        emu_launch((nb * nfq + 7) / 8, 256, 0, [&] {
            smm::beta_kernel(nb, nd, n, p, nfq, s.bface_elem.data(), s.bface_face.data(), s.quad.w.data(),
                             s.quad.ox.data(), s.quad.oy.data(), s.L1.data(), s.b_nhat.data(), s.b_eb0.data(),
                             psi.data(), mom.data(), beta.data());
        });
    std::ofstream dims(dir + "/dims.txt");
    dims << n << " " << nd << " " << nfq << " " << nb << "\n";
    const bool ok = write_file(dir + "/mom.f64", mom) && write_file(dir + "/mom_df.f64", mom_df) &&
                    write_file(dir + "/beta.f64", beta);
    return ok && dims ? 0 : 5;
}
