// Test driver (CPU): the wavefront sweep kernel of sweep.cu run on the host
// through host_kernel_shim.h, in both FP64 local-solve forms the library
// launches in source mode: the in-register LU (sweep_kernel<double, P,
// SWEEP_SOURCE, false>) and the cached local inverses held as FP32 pairs
// (invert_kernel, source_kernel and mass_apply_kernel first, then
// sweep_kernel<double, P, SWEEP_SOURCE, true>).  The inputs are the library's
// host setup (task list, face directions, element and face matrices) in the
// device layouts, filled as the library fills its sweep arguments.  One block
// of 256 threads (8 warps) takes the level-sorted task list round-robin, so
// the epoch-flag waits between warps are exercised with real threads.  The
// kernel source arrives as sweep_kernels.inc, extracted from the CUDA files by
// the test; the inline-assembly loads, stores and timer it wraps are given
// here as C++ atomics and a steady clock.
// MODE fixup runs the kernels with the optional parts compiled in (EXT) and
// the zero-and-scale fixup on; MODE refine runs, instead of the FP64 sweep,
// K sweeps of the FP32-refined form: residual_kernel (FP64 transport residual
// of the accumulated flux) and sweep_kernel<float, P, SWEEP_RESIDUAL> solving
// for the correction in FP32 and adding it to the FP64 flux (the LU form, and
// the cached FP32 inverses from invert_kernel<float, P>).
// MODE timeout first runs each form with the first task of the list left out,
// so the flag of that task is never published and the tasks downwind of it
// wait until the bounded wait gives up (timeout 20 ms): the kernel must
// return with the device error word set to DEV_TIMEOUT, every warp having
// stopped.  It then sweeps again with the next flag epoch and the whole list,
// as the library's next sweep does, and that sweep's flux is the output.  The
// error words of both runs go to DIR/timeout_err.txt.
// MODE lag runs the kernels with the optional parts compiled in on a mesh whose
// upwind graphs have cycles: the faces the setup lagged read DIR/psi_lag.f64
// ([ne][nd][n], the previous sweep's flux), the faces that are inflow at some
// points and outflow at others use their pointwise face matrices.
// Usage: sweep_emu DIR NE NNODES M P SN ANGULAR INFLOW MODE K   (one problem)
//        sweep_emu --batch DIR COUNT                          (see run_batch)
//   in:  DIR/nodes.f64, elem.i32, sigma_t.f64, sigma_s.f64, phi.f64 [ne][n],
//        q.f64 ([ne][n], or [nd][ne][n] if ANGULAR), inflow.f64 [nd][n_bface][p+1] if INFLOW,
//        nbface.txt (the boundary face count); MODE plain | fixup | refine | timeout | lag, K sweeps (refine)
//   out: DIR/dims.txt (n nd n_bface nlevels), DIR/psi_lu.f64, DIR/psi_inv.f64 and (FP64 modes)
//        DIR/psi2_inv.f64 (the pair copy as hi + lo) [ne][nd][n], the moments the sweep forms
//        DIR/mom_lu.f64, DIR/mom_inv.f64 [6][ne][n] and beta DIR/beta_lu.f64, DIR/beta_inv.f64
//        [n_bface][nfq], DIR/err.txt (device error words)
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "host_kernel_shim.h"
#include "setup.hpp"

namespace smm {

inline unsigned ld_acquire(const unsigned* p) {
    return std::atomic_ref<unsigned>(*const_cast<unsigned*>(p)).load(std::memory_order_acquire);
}
inline void st_release(unsigned* p, unsigned v) { std::atomic_ref<unsigned>(*p).store(v, std::memory_order_release); }
inline long long global_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}
inline int ld_volatile(const int* p) {
    return std::atomic_ref<int>(*const_cast<int*>(p)).load(std::memory_order_relaxed);
}

#include "sweep_kernels.inc"

}  // namespace smm

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

static std::vector<float2> to_pairs(const std::vector<double>& v) {
    std::vector<float2> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) out[i] = smm::df_make(v[i]);
    return out;
}

struct Run {
    std::vector<double> psi;
    std::vector<float2> psi2;
    std::vector<double> mom, beta;   // formed inside the sweep after all its tasks
    std::vector<unsigned> gate;
    std::vector<float2> wq2;
    int err = 0;
};

// the fused moments' arguments, as the library's sweep preparation fills them:
// the gate (zero), the weights (and their pair copies w_d (1, Ox, Oy, OxOx,
// OxOy, OyOy)), the boundary data, and the outputs
template <typename T>
static void moment_args(const smm::Setup& s, smm::SweepArgs<T>& a, Run& out, const double* mpsi) {
    const int ne = s.ne, nd = s.nd, n = s.n;
    out.gate.assign(1, 0u);
    out.wq2.resize((size_t)6 * nd);
    for (int d = 0; d < nd; ++d) {
        const double w = s.quad.w[d], x = s.quad.ox[d], y = s.quad.oy[d];
        const double v[6] = {w, w * x, w * y, w * x * x, w * x * y, w * y * y};
        for (int k = 0; k < 6; ++k) out.wq2[(size_t)k * nd + d] = smm::df_make(v[k]);
    }
    out.mom.assign((size_t)6 * ne * n, 0.0);
    out.beta.assign((size_t)s.nb * s.nfq, 0.0);
    a.gate = out.gate.data(); a.w = s.quad.w.data(); a.wq2 = out.wq2.data(); a.mpsi = mpsi;
    a.mom = out.mom.data(); a.beta = s.nb > 0 ? out.beta.data() : nullptr; a.nfq = s.nfq; a.L1 = s.L1.data();
    a.nhat = s.b_nhat.data(); a.eb0 = s.b_eb0.data();
}

// FP64 cached mode keeps the flux only as pairs: its FP64 value, as smm_get_psi forms it
static void pairs_to_psi(Run& r) {
    r.psi.resize(r.psi2.size());
    for (size_t i = 0; i < r.psi2.size(); ++i) r.psi[i] = (double)r.psi2[i].x + (double)r.psi2[i].y;
}

// the arguments the library's sweep preparation fills for an FP64 source sweep
static smm::SweepArgs<double> base_args(const smm::Setup& s, const std::vector<double>& phi, bool inflow,
                                        std::vector<unsigned>& done, int& err) {
    smm::SweepArgs<double> a{};
    a.ne = s.ne; a.nd = s.nd; a.ntask = (int)s.tasks.size(); a.p = s.p; a.tasks = s.tasks.data();
    a.ox = s.quad.ox.data(); a.oy = s.quad.oy.data(); a.sigma_t = s.sigma_t.data(); a.sigma_s = s.sigma_s.data();
    a.M = s.M.data(); a.Gx = s.Gx.data(); a.Gy = s.Gy.data(); a.Fx = s.Fx.data(); a.Fy = s.Fy.data();
    a.fdir = s.fdir.data(); a.nbr = s.nbr.data(); a.nbr_face = s.nbr_face.data(); a.nbr_flip = s.nbr_flip.data();
    a.bface_id = s.bface_id.data();
    a.phi = phi.data(); a.src = s.src.data(); a.src_angular = s.src.size() > (size_t)s.ne * s.n ? 1 : 0;
    a.inflow = inflow ? s.inflow.data() : nullptr;
    done.assign((size_t)s.ne * s.nd, 0u);
    a.done = done.data(); a.epoch = 1; a.err = &err;
    a.timeout_ns = 60LL * 1000 * 1000 * 1000;
    if (!s.fmix.empty()) {
        static thread_local std::vector<float2> fmix2;
        fmix2 = to_pairs(s.fmix);
        a.fmix_id = s.fmix_id.data(); a.fmix = s.fmix.data(); a.fmix2 = fmix2.data();
    }
    return a;
}

// what the library's create and sweep preparation add for the cached pair
// inverses: the inverses (invert_kernel), M s (source_kernel), M q_d for an
// angular source (mass_apply_kernel) and the pair copies of the cosines, face
// matrices and inflow
struct Cached {
    std::vector<float2> ainv, msrc, mq, ox2, oy2, Fx2, Fy2, inflow2;
};

template <int P>
static void prepare_cached(const smm::Setup& s, const std::vector<double>& phi, bool inflow,
                           smm::SweepArgs<double>& a, Cached& c) {
    const int ne = s.ne, nd = s.nd, n = s.n, ntask = a.ntask;
    const size_t nang = (size_t)ne * nd * n;
    c.ainv.resize((size_t)ntask * n * n);
    c.msrc.resize((size_t)ne * n);
    emu_launch((ntask + 7) / 8, 256, 0, [&] { smm::invert_kernel<double, P>(a, nullptr, c.ainv.data()); });
    emu_launch((ne * n + 255) / 256, 256, 0, [&] {
        smm::source_kernel(ne, n, s.M.data(), s.sigma_s.data(), phi.data(), a.src_angular ? nullptr : s.src.data(),
                           c.msrc.data());
    });
    if (a.src_angular) {
        c.mq.resize(nang);
        emu_launch((int)((nang + 255) / 256), 256, 0,
                   [&] { smm::mass_apply_kernel(ne, nd, n, s.M.data(), s.src.data(), c.mq.data()); });
    }
    c.ox2 = to_pairs(s.quad.ox); c.oy2 = to_pairs(s.quad.oy); c.Fx2 = to_pairs(s.Fx); c.Fy2 = to_pairs(s.Fy);
    c.inflow2 = to_pairs(s.inflow);
    a.ainv_df = c.ainv.data(); a.msrc2 = c.msrc.data(); a.mq2 = a.src_angular ? c.mq.data() : nullptr;
    a.ox2 = c.ox2.data(); a.oy2 = c.oy2.data(); a.Fx2 = c.Fx2.data(); a.Fy2 = c.Fy2.data();
    a.inflow2 = inflow ? c.inflow2.data() : nullptr;
}

// column sums of M, Gx, Gy and of the face matrices over their test index, as
// the library forms them for the fixup
struct ColSums {
    std::vector<double> m, gx, gy, fx, fy;
    explicit ColSums(const smm::Setup& s) {
        const int n = s.n, p1 = s.p1;
        const size_t nn = (size_t)n * n;
        m.assign((size_t)s.ne * n, 0.0); gx = m; gy = m;
        fx.assign((size_t)s.ne * 4 * p1, 0.0); fy = fx;
        for (int e = 0; e < s.ne; ++e) {
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    m[(size_t)e * n + j] += s.M[e * nn + (size_t)i * n + j];
                    gx[(size_t)e * n + j] += s.Gx[e * nn + (size_t)i * n + j];
                    gy[(size_t)e * n + j] += s.Gy[e * nn + (size_t)i * n + j];
                }
            for (int f = 0; f < 4; ++f)
                for (int a = 0; a < p1; ++a)
                    for (int b = 0; b < p1; ++b) {
                        const size_t fo = (((size_t)e * 4 + f) * p1 + a) * p1 + b;
                        fx[((size_t)e * 4 + f) * p1 + b] += s.Fx[fo];
                        fy[((size_t)e * 4 + f) * p1 + b] += s.Fy[fo];
                    }
        }
    }
    void fill(smm::SweepArgs<double>& a) const {
        a.fixup = 1;
        a.colM = m.data(); a.colGx = gx.data(); a.colGy = gy.data(); a.colFx = fx.data(); a.colFy = fy.data();
    }
};

// K sweeps of the FP32-refined form from psi = 0, both local-solve forms
template <int P>
static void run_refined(const smm::Setup& s, const std::vector<double>& phi, bool inflow, int K, Run& lu, Run& inv) {
    const int ne = s.ne, nd = s.nd, n = s.n, ntask = (int)s.tasks.size();
    const size_t nang = (size_t)ne * nd * n;
    const std::vector<float> M(s.M.begin(), s.M.end()), Gx(s.Gx.begin(), s.Gx.end()), Gy(s.Gy.begin(), s.Gy.end());
    const std::vector<float> Fx(s.Fx.begin(), s.Fx.end()), Fy(s.Fy.begin(), s.Fy.end());
    for (int form = 0; form < 2; ++form) {
        Run& out = form == 0 ? lu : inv;
        out.psi.assign(nang, 0.0);
        std::vector<float> res(nang), dpsi(nang), ainv;
        std::vector<unsigned> done((size_t)ne * nd, 0u);
        smm::SweepArgs<float> a{};
        a.ne = ne; a.nd = nd; a.ntask = ntask; a.p = s.p; a.tasks = s.tasks.data();
        a.ox = s.quad.ox.data(); a.oy = s.quad.oy.data(); a.sigma_t = s.sigma_t.data(); a.sigma_s = s.sigma_s.data();
        a.M = M.data(); a.Gx = Gx.data(); a.Gy = Gy.data(); a.Fx = Fx.data(); a.Fy = Fy.data();
        a.fdir = s.fdir.data(); a.nbr = s.nbr.data(); a.nbr_face = s.nbr_face.data(); a.nbr_flip = s.nbr_flip.data();
        a.bface_id = s.bface_id.data();
        a.rhs = res.data(); a.psi = dpsi.data(); a.psi_acc = out.psi.data();
        moment_args(s, a, out, out.psi.data());
        a.done = done.data(); a.err = &out.err;
        a.timeout_ns = 60LL * 1000 * 1000 * 1000;
        if (form == 1) {
            ainv.resize((size_t)ntask * n * n);
            emu_launch((ntask + 7) / 8, 256, 0, [&] { smm::invert_kernel<float, P>(a, ainv.data(), nullptr); });
            a.ainv = ainv.data();
        }
        smm::ResidualArgs r{};
        r.ne = ne; r.nd = nd; r.ntask = ntask; r.ox = a.ox; r.oy = a.oy; r.sigma_t = a.sigma_t; r.sigma_s = a.sigma_s;
        r.M = s.M.data(); r.Gx = s.Gx.data(); r.Gy = s.Gy.data(); r.Fx = s.Fx.data(); r.Fy = s.Fy.data();
        r.fdir = a.fdir; r.nbr = a.nbr; r.nbr_face = a.nbr_face; r.nbr_flip = a.nbr_flip; r.bface_id = a.bface_id;
        r.phi = phi.data(); r.src = s.src.data(); r.src_angular = s.src.size() > (size_t)ne * n ? 1 : 0;
        r.inflow = inflow ? s.inflow.data() : nullptr; r.psi = out.psi.data(); r.rhs = res.data();
        for (int k = 0; k < K; ++k) {
            emu_launch((ntask + 7) / 8, 256, 0, [&] { smm::residual_kernel<P>(r); });
            a.epoch = (unsigned)(k + 1);
            out.gate[0] = 0u;
            if (form == 0)
                emu_launch(1, 256, 0, [&] { smm::sweep_kernel<float, P, smm::SWEEP_RESIDUAL, false, false>(a); });
            else
                emu_launch(1, 256, 0, [&] { smm::sweep_kernel<float, P, smm::SWEEP_RESIDUAL, true, false>(a); });
        }
    }
}

template <int P>
static void run(const smm::Setup& s, const std::vector<double>& phi, bool inflow, bool fixup, Run& lu, Run& inv,
                const std::vector<double>* lag = nullptr) {
    const int ne = s.ne, nd = s.nd, n = s.n;
    const size_t nang = (size_t)ne * nd * n;
    const ColSums cols(s);
    const std::vector<float2> lag2 = lag ? to_pairs(*lag) : std::vector<float2>();
    {  // in-register LU
        std::vector<unsigned> done;
        smm::SweepArgs<double> a = base_args(s, phi, inflow, done, lu.err);
        lu.psi.assign(nang, 0.0);
        a.psi = lu.psi.data();
        moment_args(s, a, lu, lu.psi.data());
        if (lag) {
            a.psi_lag = lag->data();
            emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, false, true>(a); });
        } else if (fixup) {
            cols.fill(a);
            emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, false, true>(a); });
        } else {
            emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, false, false>(a); });
        }
    }
    {  // cached inverses as FP32 pairs
        std::vector<unsigned> done;
        smm::SweepArgs<double> a = base_args(s, phi, inflow, done, inv.err);
        Cached store;
        prepare_cached<P>(s, phi, inflow, a, store);
        inv.psi2.assign(nang, make_float2(0.0f, 0.0f));
        a.psi = nullptr; a.psi2 = inv.psi2.data();
        moment_args(s, a, inv, nullptr);
        if (lag) {
            a.psi2_lag = lag2.data();
            emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, true, true>(a); });
        } else if (fixup) {
            cols.fill(a);
            emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, true, true>(a); });
        } else {
            emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, true, false>(a); });
        }
        pairs_to_psi(inv);
    }
}

// Each form twice on the same flags: once without the list's first task (its
// flag is never published, so its downwind tasks' waits expire), then, with
// the device error word cleared and the next epoch, over the whole list.
// e1/e2: the error words after the first and the second run of each form.
template <int P>
static void run_timeout(const smm::Setup& s, const std::vector<double>& phi, bool inflow, Run& lu, Run& inv,
                        int e1[2], int e2[2]) {
    const int ne = s.ne, nd = s.nd, n = s.n;
    const size_t nang = (size_t)ne * nd * n;
    for (int form = 0; form < 2; ++form) {
        Run& out = form == 0 ? lu : inv;
        std::vector<unsigned> done;
        smm::SweepArgs<double> a = base_args(s, phi, inflow, done, out.err);
        Cached store;
        if (form == 1) prepare_cached<P>(s, phi, inflow, a, store);
        out.psi.assign(nang, 0.0);
        out.psi2.assign(nang, make_float2(0.0f, 0.0f));
        a.psi = form == 0 ? out.psi.data() : nullptr;
        if (form == 1) a.psi2 = out.psi2.data();
        moment_args(s, a, out, form == 0 ? out.psi.data() : nullptr);
        auto sweep = [&] {
            if (form == 0)
                emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, false, false>(a); });
            else
                emu_launch(1, 256, 0, [&] { smm::sweep_kernel<double, P, smm::SWEEP_SOURCE, true, false>(a); });
        };
        a.tasks = s.tasks.data() + 1;
        a.ntask = (int)s.tasks.size() - 1;
        a.timeout_ns = 20LL * 1000 * 1000;
        sweep();
        e1[form] = out.err;
        out.err = 0;
        a.tasks = s.tasks.data();
        a.ntask = (int)s.tasks.size();
        a.epoch = 2;
        a.timeout_ns = 60LL * 1000 * 1000 * 1000;
        out.gate[0] = 0u;
        sweep();
        e2[form] = out.err;
        if (form == 1) pairs_to_psi(out);
    }
}

// one problem's inputs (see the usage above) and the library's host setup of them
struct Problem {
    smm::Setup s;
    std::vector<double> phi;
    bool inflow = false;
};

static int load_problem(const std::string& dir, int ne, int nn, int m, int p, int sn, int angular, int inflow,
                        Problem& pr) {
    const int n = (p + 1) * (p + 1);
    std::vector<double> nodes((size_t)nn * 2), st(ne), ss(ne);
    std::vector<int32_t> elem((size_t)ne * (m + 1) * (m + 1));
    pr.phi.assign((size_t)ne * n, 0.0);
    pr.inflow = inflow != 0;
    if (!read_file(dir + "/nodes.f64", nodes) || !read_file(dir + "/elem.i32", elem) ||
        !read_file(dir + "/sigma_t.f64", st) || !read_file(dir + "/sigma_s.f64", ss) ||
        !read_file(dir + "/phi.f64", pr.phi))
        return 3;
    // the ordinate count and the boundary face count size the angular inputs
    const int nd = sn * (sn + 2) / 2;
    int nb = 0;
    {
        std::ifstream f(dir + "/nbface.txt");
        f >> nb;
    }
    std::vector<double> q((size_t)(angular ? nd : 1) * ne * n), infl(inflow ? (size_t)nd * nb * (p + 1) : 0);
    if (!read_file(dir + "/q.f64", q)) return 3;
    if (inflow && !read_file(dir + "/inflow.f64", infl)) return 3;
    smm::Input in;
    in.ne = ne; in.m = m; in.p = p; in.sn = sn; in.n_nodes = nn;
    in.nodes = nodes.data(); in.elem_nodes = elem.data(); in.sigma_t = st.data(); in.sigma_s = ss.data();
    in.source_kind = angular ? 1 : 0; in.q = q.data();
    in.inflow_kind = inflow ? 1 : 0; in.inflow = inflow ? infl.data() : nullptr;
    std::string err;
    if (smm::build_setup(in, pr.s, err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 4;
    }
    return pr.s.nd == nd && pr.s.nb == nb ? 0 : 6;
}

static bool write_outputs(const std::string& dir, const smm::Setup& s, const Run& lu, const Run& inv) {
    std::vector<double> psi2(inv.psi2.size());
    for (size_t i = 0; i < psi2.size(); ++i) psi2[i] = (double)inv.psi2[i].x + (double)inv.psi2[i].y;
    std::ofstream dims(dir + "/dims.txt");
    dims << s.n << " " << s.nd << " " << s.nb << " " << s.nlevels << "\n";
    std::ofstream errs(dir + "/err.txt");
    errs << lu.err << " " << inv.err << "\n";
    return write_file(dir + "/psi_lu.f64", lu.psi) && write_file(dir + "/psi_inv.f64", inv.psi) &&
           write_file(dir + "/psi2_inv.f64", psi2) && write_file(dir + "/mom_lu.f64", lu.mom) &&
           write_file(dir + "/mom_inv.f64", inv.mom) && write_file(dir + "/beta_lu.f64", lu.beta) &&
           write_file(dir + "/beta_inv.f64", inv.beta) && (bool)dims && (bool)errs;
}

// sweep_emu --batch DIR COUNT: problems DIR/0 .. DIR/COUNT-1 (each with its
// inputs and args.txt = "NE NNODES M P SN ANGULAR INFLOW") swept together by
// batch_sweep_kernel over their merged task list (level by level, problem by
// problem, as the library merges it), with the LU and with cached inverses
static int run_batch(const std::string& dir, int count) {
    std::vector<Problem> prs(count);
    for (int k = 0; k < count; ++k) {
        const std::string d = dir + "/" + std::to_string(k);
        std::ifstream f(d + "/args.txt");
        int ne, nn, m, p, sn, ang, infl;
        if (!(f >> ne >> nn >> m >> p >> sn >> ang >> infl)) return 3;
        const int rc = load_problem(d, ne, nn, m, p, sn, ang, infl, prs[k]);
        if (rc) return rc;
    }
    std::vector<int2> merged;
    int maxlev = 0;
    for (const Problem& pr : prs) maxlev = std::max(maxlev, pr.s.nlevels);
    for (int l = 0; l < maxlev; ++l)
        for (int k = 0; k < count; ++k) {
            const smm::Setup& s = prs[k].s;
            if (l >= s.nlevels) continue;
            for (int t = s.level_start[l]; t < s.level_start[l + 1]; ++t) merged.push_back(make_int2(k, s.tasks[t]));
        }
    std::vector<Run> lu(count), inv(count);
    for (int form = 0; form < 2; ++form) {
        std::vector<smm::SweepArgs<double>> args(count);
        std::vector<std::vector<unsigned>> done(count);
        std::vector<Cached> store(count);
        for (int k = 0; k < count; ++k) {
            const smm::Setup& s = prs[k].s;
            Run& out = form == 0 ? lu[k] : inv[k];
            args[k] = base_args(s, prs[k].phi, prs[k].inflow, done[k], out.err);
            const size_t nang = (size_t)s.ne * s.nd * s.n;
            out.psi.assign(nang, 0.0);
            args[k].psi = form == 0 ? out.psi.data() : nullptr;
            moment_args(s, args[k], out, form == 0 ? out.psi.data() : nullptr);
            if (form == 1) {
                switch (s.p) {
                    case 1: prepare_cached<1>(s, prs[k].phi, prs[k].inflow, args[k], store[k]); break;
                    case 2: prepare_cached<2>(s, prs[k].phi, prs[k].inflow, args[k], store[k]); break;
                    case 3: prepare_cached<3>(s, prs[k].phi, prs[k].inflow, args[k], store[k]); break;
                    default: prepare_cached<4>(s, prs[k].phi, prs[k].inflow, args[k], store[k]); break;
                }
                out.psi2.assign(nang, make_float2(0.0f, 0.0f));
                args[k].psi2 = out.psi2.data();
            }
        }
        const int ntask = (int)merged.size();
        // every problem's elements; one gate for the launch
        std::vector<int2> elems;
        for (int k = 0; k < count; ++k)
            for (int e = 0; e < prs[k].s.ne; ++e) elems.push_back(make_int2(k, e));
        std::vector<unsigned> gate(1, 0u);
        for (int k = 0; k < count; ++k) args[k].gate = gate.data();
        const int nelem = (int)elems.size();
        if (form == 0)
            emu_launch(1, 256, 0, [&] {
                smm::batch_sweep_kernel<double, smm::SWEEP_SOURCE, false, false, 4>(args.data(), merged.data(), ntask,
                                                                          elems.data(), nelem);
            });
        else
            emu_launch(1, 256, 0, [&] {
                smm::batch_sweep_kernel<double, smm::SWEEP_SOURCE, true, false, 4>(args.data(), merged.data(), ntask,
                                                                         elems.data(), nelem);
            });
    }
    for (int k = 0; k < count; ++k) {
        pairs_to_psi(inv[k]);
        if (!write_outputs(dir + "/" + std::to_string(k), prs[k].s, lu[k], inv[k])) return 5;
    }
    return 0;
}

int main(int argc, char** argv) {
    if (argc == 4 && std::string(argv[1]) == "--batch") return run_batch(argv[2], std::atoi(argv[3]));
    if (argc != 11) return 2;
    const std::string mode = argv[9];
    const int K = std::atoi(argv[10]);
    if (mode != "plain" && mode != "fixup" && mode != "refine" && mode != "timeout" && mode != "lag") return 2;
    const std::string dir = argv[1];
    const int ne = std::atoi(argv[2]), nn = std::atoi(argv[3]), m = std::atoi(argv[4]), p = std::atoi(argv[5]);
    const int sn = std::atoi(argv[6]), angular = std::atoi(argv[7]), inflow = std::atoi(argv[8]);
    Problem pr;
    const int rc = load_problem(dir, ne, nn, m, p, sn, angular, inflow, pr);
    if (rc) return rc;
    const smm::Setup& s = pr.s;
    Run lu, inv;
    const bool fix = mode == "fixup";
    if (mode == "timeout") {
        int e1[2] = {0, 0}, e2[2] = {0, 0};
        switch (p) {
            case 1: run_timeout<1>(s, pr.phi, pr.inflow, lu, inv, e1, e2); break;
            case 2: run_timeout<2>(s, pr.phi, pr.inflow, lu, inv, e1, e2); break;
            case 3: run_timeout<3>(s, pr.phi, pr.inflow, lu, inv, e1, e2); break;
            default: run_timeout<4>(s, pr.phi, pr.inflow, lu, inv, e1, e2); break;
        }
        std::ofstream f(dir + "/timeout_err.txt");
        f << e1[0] << " " << e2[0] << " " << e1[1] << " " << e2[1] << "\n";
    } else if (mode == "refine") {
        switch (p) {
            case 1: run_refined<1>(s, pr.phi, pr.inflow, K, lu, inv); break;
            case 2: run_refined<2>(s, pr.phi, pr.inflow, K, lu, inv); break;
            case 3: run_refined<3>(s, pr.phi, pr.inflow, K, lu, inv); break;
            default: run_refined<4>(s, pr.phi, pr.inflow, K, lu, inv); break;
        }
    } else {
        std::vector<double> lagv;
        if (mode == "lag") {
            lagv.resize((size_t)s.ne * s.nd * s.n);
            if (!read_file(dir + "/psi_lag.f64", lagv)) return 3;
        }
        const std::vector<double>* lag = mode == "lag" ? &lagv : nullptr;
        switch (p) {
            case 1: run<1>(s, pr.phi, pr.inflow, fix, lu, inv, lag); break;
            case 2: run<2>(s, pr.phi, pr.inflow, fix, lu, inv, lag); break;
            case 3: run<3>(s, pr.phi, pr.inflow, fix, lu, inv, lag); break;
            default: run<4>(s, pr.phi, pr.inflow, fix, lu, inv, lag); break;
        }
    }
    return write_outputs(dir, s, lu, inv) ? 0 : 5;
}
