// Test driver (CPU): runs the library's host setup and multigrid hierarchy
// construction on a mesh read from files, the way smm_create calls them, and
// writes the hierarchy.  Usage: mg_dump DIR NE NNODES M P COARSE_MAX
//   in:  as setup_dump (DIR/nodes.f64, elem.i32, sigma_t.f64, q.f64)
//   out: DIR/mg.txt: "nvert ncoarse nlevels omega0", then per level l >= 1 "nrow omega has_P";
//        DIR/{Adiag,Aoff,Pinv}.f64 (the level-0 blocks), DIR/nbr.i32, DIR/vid.i32 [ne][4], DIR/w4.f64 [n][4],
//        DIR/vrp.i32, DIR/vinc.i32, DIR/coarse_inv.f64, and per level l >= 1 DIR/L<l>_{A,P,R}_{rp,ci}.i32,
//        DIR/L<l>_{A,P,R}_v.f64, DIR/L<l>_dinv.f64 (P and R only where has_P).
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "amg.hpp"
#include "setup.hpp"

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

static bool write_csr(const std::string& stem, const smm::CSR& A) {
    return write_file(stem + "_rp.i32", A.rp) && write_file(stem + "_ci.i32", A.ci) && write_file(stem + "_v.f64", A.v);
}

int main(int argc, char** argv) {
    if (argc != 7) return 2;
    const std::string dir = argv[1];
    const int ne = std::atoi(argv[2]), nn = std::atoi(argv[3]), m = std::atoi(argv[4]), p = std::atoi(argv[5]);
    const int coarse_max = std::atoi(argv[6]);
    const int n = (p + 1) * (p + 1), nc = (m + 1) * (m + 1);
    std::vector<double> nodes((size_t)nn * 2), st(ne), ss(ne), q((size_t)ne * n);
    std::vector<int32_t> elem((size_t)ne * nc);
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
    std::vector<int> corners((size_t)ne * 4);
    const int cidx[4] = {0, m, m * (m + 1), m * (m + 1) + m};
    for (int e = 0; e < ne; ++e)
        for (int c = 0; c < 4; ++c) corners[(size_t)e * 4 + c] = elem[(size_t)e * nc + cidx[c]];
    std::vector<int> nbr(s.nbr.begin(), s.nbr.end());
    smm::MGHierarchy H;
    if (!smm::build_multigrid(ne, n, s.Adiag, s.Aoff, s.Pinv, nbr, corners, smm::gauss_lobatto01(p + 1).x, H, err,
                              coarse_max)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    std::ofstream txt(dir + "/mg.txt");
    txt.precision(17);
    txt << H.nvert << " " << H.ncoarse << " " << H.lv.size() - 1 << " " << H.omega0 << "\n";
    bool ok = write_file(dir + "/Adiag.f64", s.Adiag) && write_file(dir + "/Aoff.f64", s.Aoff) &&
              write_file(dir + "/Pinv.f64", s.Pinv) && write_file(dir + "/nbr.i32", nbr) &&
              write_file(dir + "/vid.i32", H.vid) && write_file(dir + "/w4.f64", H.w4) &&
              write_file(dir + "/vrp.i32", H.vrp) && write_file(dir + "/vinc.i32", H.vinc) &&
              write_file(dir + "/coarse_inv.f64", H.coarse_inv);
    for (size_t l = 1; l < H.lv.size(); ++l) {
        const smm::MGLevel& L = H.lv[l];
        const bool hasP = L.P.nrow > 0;
        txt << L.A.nrow << " " << L.omega << " " << (hasP ? 1 : 0) << "\n";
        const std::string stem = dir + "/L" + std::to_string(l);
        ok = ok && write_csr(stem + "_A", L.A) && write_file(stem + "_dinv.f64", L.dinv);
        if (hasP) ok = ok && write_csr(stem + "_P", L.P) && write_csr(stem + "_R", L.R);
    }
    return ok && txt ? 0 : 5;
}
