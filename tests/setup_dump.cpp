// Test driver (CPU): runs the library's host setup on a mesh read from files
// and writes the element operators it builds, so that a test can compare them
// with the oracle.  Usage: setup_dump DIR NE NNODES M P
//   in:  DIR/nodes.f64 [nnodes][2], DIR/elem.i32 [ne][(m+1)^2], DIR/sigma_t.f64 [ne],
//        DIR/q.f64 [ne][n] isotropic source per steradian (sigma_s = sigma_t / 2)
//   a sixth argument "nolag" turns cycle lagging off
//   out: DIR/dims.txt (n nfq nd nlevels), DIR/{Kxx,Ks,Kyy,Dfx,Dfy,nds,M,Gx,Gy,Adiag,Aoff,Pinv,bfixed,
//        ox,oy,w}.f64, DIR/{nbr,level,tasks,level_start}.i32, DIR/fdir.i8 [ne][nd][4]
//   A setup error is printed on stderr and gives exit status 4.
//   setup_dump --size-check NE M P SN: see size_check below.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

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

// setup_dump --size-check NE M P SN: build_setup on NE elements whose arrays
// are never read (one-element stand-ins); exit status 4 with the message on
// stderr when the setup rejects the size before it touches them.
static int size_check(int ne, int m, int p, int sn) {
    std::vector<double> one(1, 1.0);
    std::vector<int32_t> zero(1, 0);
    smm::Input in;
    in.ne = ne; in.m = m; in.p = p; in.sn = sn; in.n_nodes = 1;
    in.nodes = one.data(); in.elem_nodes = zero.data(); in.sigma_t = one.data(); in.sigma_s = one.data();
    in.q = one.data();
    smm::Setup s;
    std::string err;
    if (smm::build_setup(in, s, err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    return 0;
}

int main(int argc, char** argv) {
    if (argc == 6 && std::string(argv[1]) == "--size-check")
        return size_check(std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]), std::atoi(argv[5]));
    if (argc != 6 && argc != 7) return 2;
    const std::string dir = argv[1];
    const bool lag = !(argc == 7 && std::string(argv[6]) == "nolag");
    const int ne = std::atoi(argv[2]), nn = std::atoi(argv[3]), m = std::atoi(argv[4]), p = std::atoi(argv[5]);
    const int n = (p + 1) * (p + 1);
    std::vector<double> nodes((size_t)nn * 2), st(ne), ss(ne), q((size_t)ne * n, 0.0);
    std::vector<int32_t> elem((size_t)ne * (m + 1) * (m + 1));
    if (!read_file(dir + "/nodes.f64", nodes) || !read_file(dir + "/elem.i32", elem) ||
        !read_file(dir + "/sigma_t.f64", st) || !read_file(dir + "/q.f64", q))
        return 3;
    for (int e = 0; e < ne; ++e) ss[e] = 0.5 * st[e];
    smm::Input in;
    in.ne = ne; in.m = m; in.p = p; in.sn = 4; in.n_nodes = nn;
    in.nodes = nodes.data(); in.elem_nodes = elem.data(); in.sigma_t = st.data(); in.sigma_s = ss.data();
    in.q = q.data();
    in.lag_cycles = lag ? 1 : 0;
    smm::Setup s;
    std::string err;
    if (smm::build_setup(in, s, err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    std::ofstream dims(dir + "/dims.txt");
    dims << s.n << " " << s.nfq << " " << s.nd << " " << s.nlevels << "\n";
    const bool ok = write_file(dir + "/Kxx.f64", s.Kxx) && write_file(dir + "/Ks.f64", s.Ks) &&
                    write_file(dir + "/Kyy.f64", s.Kyy) && write_file(dir + "/Dfx.f64", s.Dfx) &&
                    write_file(dir + "/Dfy.f64", s.Dfy) && write_file(dir + "/nds.f64", s.nds) &&
                    write_file(dir + "/M.f64", s.M) && write_file(dir + "/Gx.f64", s.Gx) &&
                    write_file(dir + "/Gy.f64", s.Gy) && write_file(dir + "/Adiag.f64", s.Adiag) &&
                    write_file(dir + "/Aoff.f64", s.Aoff) && write_file(dir + "/Pinv.f64", s.Pinv) &&
                    write_file(dir + "/bfixed.f64", s.bfixed) && write_file(dir + "/ox.f64", s.quad.ox) &&
                    write_file(dir + "/oy.f64", s.quad.oy) && write_file(dir + "/w.f64", s.quad.w) &&
                    write_file(dir + "/nbr.i32", s.nbr) && write_file(dir + "/level.i32", s.level) &&
                    write_file(dir + "/tasks.i32", s.tasks) && write_file(dir + "/level_start.i32", s.level_start) &&
                    write_file(dir + "/fdir.i8", s.fdir);
    return ok ? 0 : 5;
}
