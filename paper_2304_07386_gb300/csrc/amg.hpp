// Multigrid hierarchy for the IP-SMM moment operator (host construction).
//
// Level 0 is the DG-p operator itself (n x n element blocks), smoothed by
// damped element-block Jacobi.  Level 1 is its Galerkin restriction to the
// continuous, mapped bilinear functions on the mesh vertices (a conforming
// subspace of Y_p: a DG-p nodal value is the reference-bilinear interpolant
// of the element's four corner values), A1 = P1^T A P1.  Further levels come
// from smoothed aggregation: strength-based aggregates, tentative
// piecewise-constant prolongator smoothed by one damped Jacobi step,
// Galerkin products.  The coarsest level is inverted densely.
#pragma once

#include <string>
#include <vector>

namespace smm {

struct CSR {
    int nrow = 0, ncol = 0;
    std::vector<int> rp, ci;
    std::vector<double> v;
};

struct MGLevel {
    CSR A;                      // operator on this level (levels >= 1)
    CSR P, R;                   // prolongation from level l+1 and its transpose (R = P^T)
    std::vector<double> dinv;   // 1 / diag(A)
    double omega = 0.0;         // Jacobi damping
};

struct MGHierarchy {
    double omega0 = 0.0;              // damping of the level-0 block-Jacobi smoother
    int nvert = 0;                    // level-1 unknowns (mesh vertices)
    std::vector<int> vid;             // [ne][4] vertex of each element corner (c00, c10, c01, c11)
    std::vector<double> w4;           // [n][4] bilinear weights of the DG-p nodes
    std::vector<int> vrp, vinc;       // vertex -> incident (element*4 + corner), CSR
    std::vector<MGLevel> lv;          // lv[0] unused placeholder; lv[1] = vertex bilinear space, ...
    std::vector<double> coarse_inv;   // dense inverse of the coarsest operator, row-major
    int ncoarse = 0;
};

// Adiag/Aoff/Pinv: row-major blocks as in Setup (Aoff empty: no neighbour
// blocks, as for the continuous-space operator; Pinv empty: no level-0
// block-Jacobi damping estimate, omega0 stays 0); nbr [ne][4]; corner_ids
// [ne][4] control-point ids of the element corners (c00, c10, c01, c11);
// gll: the p+1 Gauss-Lobatto points of [0,1].
bool build_multigrid(int ne, int n, const std::vector<double>& Adiag, const std::vector<double>& Aoff,
                     const std::vector<double>& Pinv, const std::vector<int>& nbr, const std::vector<int>& corner_ids,
                     const std::vector<double>& gll, MGHierarchy& mg, std::string& err, int coarse_max = 400);

}  // namespace smm
