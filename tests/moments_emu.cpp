// Test driver (CPU): the moment epilogue of the sweep kernel (element_moments
// in sweep.cu: the angular moments from the FP64 flux, or from its FP32-pair
// copy as in FP64 cached mode, and beta at the boundary Gauss points) run on
// the host through host_kernel_shim.h, one warp per element (as after the
// sweep's gate, every ordinate already swept), on the quadrature and boundary data the
// library's host setup builds, in the library's layouts.  The function's
// source arrives as moments_kernels.inc, extracted from sweep.cu by the test.
// Usage: moments_emu DIR NE NNODES M P SN
//   in:  DIR/nodes.f64, elem.i32, sigma_t.f64, q.f64 (as setup_dump),
//        DIR/psi.f64 [ne][nd][n] (the device layout)
//   out: DIR/dims.txt (n nd nfq n_bface), DIR/mom.f64 and DIR/mom_df.f64 [6][ne][n],
//        DIR/beta.f64 and DIR/beta_df.f64 [n_bface][nfq]
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "host_kernel_shim.h"
#include "setup.hpp"

#include <atomic>
#include <chrono>

namespace smm {

inline unsigned ld_acquire(const unsigned* p) {
    return std::atomic_ref<unsigned>(*const_cast<unsigned*>(p)).load(std::memory_order_acquire);
}
inline long long global_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}
inline int ld_volatile(const int* p) {
    return std::atomic_ref<int>(*const_cast<int*>(p)).load(std::memory_order_relaxed);
}

#include "moments_kernels.inc"

}  // namespace smm

// every element's epilogue, one warp per element (8 warps take the elements round-robin)
template <int P, bool DF>
static void run_epilogue(const smm::SweepArgs<double>& a) {
    emu_launch(1, 256, 0, [&] {
        const int W = (gridDim.x * blockDim.x) >> 5;
        const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        for (int e = gw; e < a.ne; e += W) smm::element_moments<double, P, DF>(a, e);
    });
}

template <bool DF>
static void run_p(int p, const smm::SweepArgs<double>& a) {
    switch (p) {
        case 1: run_epilogue<1, DF>(a); break;
        case 2: run_epilogue<2, DF>(a); break;
        case 3: run_epilogue<3, DF>(a); break;
        default: run_epilogue<4, DF>(a); break;
    }
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
    std::vector<double> mom((size_t)6 * ne * n, 0.0), mom_df((size_t)6 * ne * n, 0.0);
    std::vector<double> beta((size_t)nb * nfq, 0.0), beta_df((size_t)nb * nfq, 0.0);
    smm::SweepArgs<double> a{};
    a.ne = ne; a.nd = nd; a.p = p; a.ox = s.quad.ox.data(); a.oy = s.quad.oy.data();
    a.nbr = s.nbr.data(); a.bface_id = s.bface_id.data();
    a.w = s.quad.w.data(); a.wq2 = wq.data(); a.nfq = nfq; a.L1 = s.L1.data(); a.nhat = s.b_nhat.data();
    a.eb0 = s.b_eb0.data();
    a.mpsi = psi.data(); a.mom = mom.data(); a.beta = nb > 0 ? beta.data() : nullptr;
    run_p<false>(p, a);
    a.psi2 = psi2.data(); a.mom = mom_df.data(); a.beta = nb > 0 ? beta_df.data() : nullptr;
    run_p<true>(p, a);
    std::ofstream dims(dir + "/dims.txt");
    dims << n << " " << nd << " " << nfq << " " << nb << "\n";
    const bool ok = write_file(dir + "/mom.f64", mom) && write_file(dir + "/mom_df.f64", mom_df) &&
                    write_file(dir + "/beta.f64", beta) && write_file(dir + "/beta_df.f64", beta_df);
    return ok && dims ? 0 : 5;
}
