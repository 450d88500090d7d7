// Host-side setup of the SMM solver: quadrature, mapped Q_p elements on
// curved quads, per-element sweep matrices, upwind ordering, and the
// interior penalty SMM operator blocks.  Plain C++17, no CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace smm {

struct Rule1D {
    std::vector<double> x, w;
};

// Gauss-Legendre / Gauss-Lobatto rules on [0,1].
Rule1D gauss_legendre01(int n);
Rule1D gauss_lobatto01(int n);

struct Quadrature {
    int nd = 0;
    std::vector<double> ox, oy, w;
};

// Level-symmetric LQ_N 2D set (weights sum to 4 pi); false if N unsupported.
bool level_symmetric(int N, Quadrature& q);

struct Input {
    int ne = 0, m = 1, p = 1, sn = 4, n_nodes = 0;
    const double* nodes = nullptr;       // [n_nodes][2]
    const int32_t* elem_nodes = nullptr; // [ne][(m+1)^2]
    const double* sigma_t = nullptr;     // [ne]
    const double* sigma_s = nullptr;     // [ne]
    int source_kind = 0;                 // 0 isotropic [ne][n], 1 angular [nd][ne][n]
    const double* q = nullptr;
    int inflow_kind = 0;                 // 0 vacuum, 1 nodal [nd][nb][p+1]
    const double* inflow = nullptr;
    double kappa_scale = 1.0;
    int moment_cg = 0;                   // also build the continuous (CG) moment system
    int sweep_tiles = 1;                 // parallel block Jacobi sweep over tiles x tiles tiles (1: exact)
    int lag_cycles = 1;                  // lag cycles of the upwind graphs (0: a cycle is an error)
};

struct Setup {
    int ne = 0, m = 1, p = 1, p1 = 2, n = 4, nq = 0, nqv = 0, nfq = 0, nd = 0, nb = 0;
    int nlevels = 0;
    Quadrature quad;
    // connectivity [ne][4]
    std::vector<int32_t> nbr, nbr_face, nbr_flip, bface_id;
    std::vector<int32_t> bface_elem, bface_face;  // [nb]
    // sweep data
    std::vector<double> sigma_t, sigma_s;
    std::vector<double> M, Gx, Gy;                // [ne][n][n], row = test function
    std::vector<double> Fx, Fy;                   // [ne][4][p1][p1]
    // faces that are inflow at some quadrature points and outflow at others for
    // an ordinate (fdir 2, or 3 when lagged): the id of their pair of pointwise
    // face matrices [ne][nd][4] (-1 for other faces), and the pairs
    // fmix[id][0][a][b] = sum_q max(Omega.n ds w, 0) l_a l_b (outflow part, in A)
    // and fmix[id][1][a][b] = the same with min (inflow part, on the upwind trace)
    std::vector<int32_t> fmix_id;
    std::vector<double> fmix;
    int64_t n_mixed = 0, n_cycle_lagged = 0;     // (element, ordinate, face) counts
    std::vector<int8_t> fdir;                     // [ne][nd][4]: +1 out, -1 in, -2 in from another tile
                                                  // (lagged: previous sweep's values), 0 none
    std::vector<int32_t> tile;                    // [ne] tile of the block Jacobi sweep (all 0: exact sweep)
    std::vector<int32_t> level;                   // [nd][ne]
    std::vector<int32_t> tasks;                   // e*nd + d sorted by (level, e, d)
    std::vector<int32_t> level_start;             // [nlevels+1] offsets into tasks
    std::vector<double> src;                      // [ne][nd][n] or [ne][n] (isotropic), per steradian
    std::vector<double> inflow;                   // [nb][nd][p1] (empty = vacuum)
    // face quadrature shared data
    std::vector<double> L1;                       // [nfq][p1]
    // boundary quadrature data
    std::vector<double> b_nhat;                   // [nb][nfq][2]
    std::vector<double> b_ds;                     // [nb][nfq]
    std::vector<double> b_eb0;                    // [nb][nfq]
    // moment system
    std::vector<double> Adiag, Aoff, Pinv;        // [ne][n][n], [ne][4][n][n], [ne][n][n]
    // Face-factored neighbour blocks: Aoff[e][f] = E_f^T Cface[e][f] E_f2 with
    // E_f (2(p+1) x n) = [trace at the p+1 face nodes; reference derivative
    // sum_t wd[t] u(line t) along the p+1 node lines normal to face f]
    std::vector<double> Cface;                    // [ne][4][2p1][2p1], row = own face datum
    std::vector<double> wd;                       // [p1]: l'_t(0) of the 1D GLL basis
    std::vector<double> Kxx, Ks, Kyy;             // [ne][n][n], scaled by -1/sigma_t
    std::vector<double> Dfx, Dfy;                 // [ne][4][nfq][n]
    std::vector<double> nds;                      // [ne][4][nfq][2]
    std::vector<double> bfixed;                   // [ne][n]
    std::vector<double> hK, area;
    // continuous (CG) moment system, Sec. 5.1 (built when Input::moment_cg):
    // element blocks D (Kxx + Kyy) + sigma_a M + Marshak boundary terms, the
    // global node of every element node (element nodes identified across
    // faces), the element nodes of every global node (CSR, element order) and
    // the first of them
    std::vector<double> Kcg;                      // [ne][n][n]
    std::vector<int32_t> gid;                     // [ne][n]
    int nglob = 0;
    std::vector<int32_t> grp, ginc, gown;         // [nglob+1], [ne*n], [nglob]
};

// Node of element-local index (face f, face position a, line position t):
// t = 0 is the face node, t grows into the element.
inline int face_line_node(int p, int f, int a, int t) {
    const int k = p + 1;
    switch (f) {
        case 0: return t * k + a;
        case 1: return a * k + p - t;
        case 2: return (p - t) * k + a;
        default: return a * k + t;
    }
}

// Status codes match smm_status in include/smm.h.
int build_setup(const Input& in, Setup& s, std::string& err);

}  // namespace smm
