// C ABI of liblsamg (declared in include/lsamg.h): set-up orchestration over levels,
// the preconditioner application, the FP64 PCG / flexible CG(1) driver, the adjoint
// element gradient, statistics and read-back queries.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "impl.cuh"
#include "ozaki.cuh"

namespace lsamg {
extern int g_prof_level;

namespace {

thread_local std::string g_last_error;

template <class F>
int guarded(F &&f) {
    try {
        f();
        g_last_error.clear();
        return LSAMG_OK;
    } catch (const Failure &e) {
        g_last_error = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return LSAMG_CUDA;
    } catch (...) {
        g_last_error = "unknown failure";
        return LSAMG_CUDA;
    }
}

}  // namespace

void set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {

double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

const char *kStages[] = {"validate+factor", "aggregate", "closure", "local spectral", "colour",
                         "smoother", "coarse gram", "coarsest", "other"};

__global__ void k_level0_maps(const int32_t *dofs, int64_t ne, int nT, int64_t *eptr,
                              int32_t *eidx, int64_t *aoff) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        eptr[e] = e * nT;
        aoff[e] = e * (int64_t)nT * nT;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ne * nT;
         j += (int64_t)gridDim.x * blockDim.x)
        eidx[j] = dofs[j];
}

// A_T = coef_e * (K_e + K_e^T) / 2: the symmetric part (bit-identical for symmetric input), so
// that the assemblies may read A_T column by column
__global__ void k_scale_mats(const double *mats, const double *coef, int64_t ne, int nT, double *out) {
    const int64_t sz = (int64_t)nT * nT;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ne * sz;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = j / sz;
        const int t = (int)(j - e * sz), r = t / nT, c = t % nT;
        const double *K = mats + e * sz;
        const double c0 = coef ? coef[e] : 1.0;
        out[j] = c0 * (0.5 * (K[r * nT + c] + K[c * nT + r]));
    }
}

__global__ void k_max_i32v(const int32_t *a, int64_t n, int *out) {
    int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, a[i]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_nan_check(const double *v, int64_t n, int *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) *flag = 1;
}

int32_t device_max(const int32_t *a, int64_t n, cudaStream_t s) {
    DBuf<int> o;
    o.alloc(1, s);
    o.zero(s);
    if (n > 0) {
        k_max_i32v<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 1184), 256, 0, s>>>(a, n, o.p);
        CK_LAUNCH();
    }
    return read1(o.p, s);
}

void finish_level_info(Level &L, cudaStream_t s) {
    L.max_grows_cached = device_max(L.grows.p, L.ne, s);
    if (!L.coarsest && L.nagg > 0) L.Omega_total = read1(L.Optr.p + L.nagg, s);
    // algorithmic bytes: every stored G_T entry, element map and vector entry touched once
    auto gr = to_host(L.grows.p, L.ne, s);
    auto ep = to_host(L.eptr.p, L.ne + 1, s);
    double gent = 0.0, ment = 0.0;
    for (int64_t e = 0; e < L.ne; e++) {
        gent += (double)gr[e] * (double)(ep[e + 1] - ep[e]);
        ment += (double)(ep[e + 1] - ep[e]);
    }
    L.spmv_fmas = 2.0 * gent;
    for (int t = 0; t < 2; t++) {
        const double w = t ? 8.0 : 4.0;
        L.spmv_bytes[t] = gent * w + ment * 4.0 + 3.0 * (double)L.n * w;
        L.coarse_bytes[t] = L.coarsest ? 2.0 * (double)L.n * (double)(L.n + 1) / 2.0 * w : 0.0;
    }
    if (L.coarsest)
        wave_setup(L, {{(int32_t)L.n}}, {{0}}, {(int32_t)L.n}, L.tri_cb, s);
    if (!L.coarsest && L.nagg > 0 && L.ncol > 0) {
        auto oep = to_host(L.oeptr.p, L.nagg + 1, s);
        auto oei = to_host(L.oeidx.p, oep[L.nagg], s);
        auto cag = to_host(L.colagg.p, L.nagg, s);
        for (int t = 0; t < 2; t++) L.sweep_bytes[t].assign(L.ncol, 0.0);
        L.colmax.assign(L.ncol, 0);
        L.colpairs.assign(L.ncol + 1, 0);
        std::vector<int32_t> pa;
        std::vector<int64_t> pe;
        for (int c = 0; c < L.ncol; c++) {
            for (int64_t q = L.colptr[c]; q < L.colptr[c + 1]; q++) {
                const int32_t a = cag[q];
                L.colmax[c] = std::max(L.colmax[c], L.h_nO[a]);
                for (int64_t j = oep[a]; j < oep[a + 1]; j++) {
                    pa.push_back(a);
                    pe.push_back(j);
                }
            }
            L.colpairs[c + 1] = (int64_t)pa.size();
        }
        upload(L.pair_agg, pa, s);
        upload(L.pair_ent, pe, s);
        // wavefront solve groups: each colour, then all subdomains (additive smoother)
        std::vector<std::vector<int32_t>> gs(L.ncol + 1), gid(L.ncol + 1);
        for (int c = 0; c < L.ncol; c++)
            for (int64_t q = L.colptr[c]; q < L.colptr[c + 1]; q++) {
                gs[c].push_back(L.h_nO[cag[q]]);
                gid[c].push_back(cag[q]);
                gs[L.ncol].push_back(L.h_nO[cag[q]]);
                gid[L.ncol].push_back(cag[q]);
            }
        wave_setup(L, gs, gid, L.h_nO, L.tri_cb, s);
        for (int c = 0; c < L.ncol; c++)
            for (int64_t q = L.colptr[c]; q < L.colptr[c + 1]; q++) {
                const int32_t a = cag[q];
                const double nO = L.h_nO[a];
                double g = 0.0, idx = nO;
                for (int64_t j = oep[a]; j < oep[a + 1]; j++) {
                    const int32_t e = oei[j];
                    g += (double)gr[e] * (double)(ep[e + 1] - ep[e]);
                    idx += 2.0 * (double)(ep[e + 1] - ep[e]);
                }
                for (int t = 0; t < 2; t++) {
                    const double w = t ? 8.0 : 4.0;
                    // packed factor read by both substitutions, element G blocks, index maps,
                    // residual gather / x update / residual scatter
                    L.sweep_bytes[t][c] += nO * (nO + 1) * w + g * w + idx * 4.0 + 4.0 * nO * w;
                }
            }
    }
}

void do_setup(Handle &H, const lsamg_problem *P, const lsamg_options &o) {
    cudaStream_t s = H.stream;
    double t0 = now();
    auto &st = H.stats;
    memset(&st, 0, sizeof st);
    if (!P || P->n_dofs <= 0 || P->n_elems < 0 || P->n_T <= 0 || !P->elem_dofs || !P->elem_mats)
        fail(LSAMG_INVALID_ARG, "invalid problem description");
    if (P->n_dofs >= (1ll << 30)) fail(LSAMG_LIMIT, "more than 2^30 DOFs");
    if (o.max_levels < 1 || o.max_levels > 8) fail(LSAMG_INVALID_ARG, "max_levels must be in 1..8");
    if (o.sweep_block < 0 || o.sweep_block > 64) fail(LSAMG_INVALID_ARG, "sweep_block must be in 0..64");
    if (o.smoother != 0 && o.smoother != 1) fail(LSAMG_INVALID_ARG, "smoother must be 0 or 1");
    if (o.closure != 0 && o.closure != 1) fail(LSAMG_INVALID_ARG, "closure must be 0 (G-row) or 1 (A)");
    H.err.alloc(2, s);
    H.err.zero(s);
    int *err = H.err.p;
    const int64_t ne = P->n_elems, nT = P->n_T, n = P->n_dofs;
    H.n0 = n;
    H.ne0 = ne;
    H.nT0 = (int32_t)nT;
    H.levels.clear();
    H.levels.emplace_back();
    Level &L0 = H.levels[0];
    L0.n = n;
    L0.ne = ne;
    L0.nnz_e = ne * nT;
    L0.max_nT = (int32_t)nT;
    // inputs (device or host) -> level-0 element maps and A_T = coef_e * K_e
    {
        DBuf<int32_t> hd;
        DBuf<double> hm, hc;
        const int32_t *dofs = P->elem_dofs;
        const double *mats = P->elem_mats, *coef = P->elem_coef;
        if (P->on_host) {
            hd.alloc(std::max<int64_t>(ne * nT, 1), s);
            hm.alloc(std::max<int64_t>(ne * nT * nT, 1), s);
            CK(cudaMemcpyAsync(hd.p, dofs, ne * nT * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(hm.p, mats, ne * nT * nT * sizeof(double), cudaMemcpyHostToDevice, s));
            dofs = hd.p;
            mats = hm.p;
            if (coef) {
                hc.alloc(std::max<int64_t>(ne, 1), s);
                CK(cudaMemcpyAsync(hc.p, coef, ne * sizeof(double), cudaMemcpyHostToDevice, s));
                coef = hc.p;
            }
        }
        L0.eptr.alloc(ne + 1, s);
        L0.eidx.alloc(std::max<int64_t>(ne * nT, 1), s);
        L0.aoff.alloc(ne + 1, s);
        unsigned g = (unsigned)std::min<int64_t>(std::max<int64_t>(cdiv(ne * nT + 1, 256), 1), 148 * 32);
        k_level0_maps<<<g, 256, 0, s>>>(dofs, ne, (int)nT, L0.eptr.p, L0.eidx.p, L0.aoff.p);
        CK_LAUNCH();
        L0.AT.alloc(std::max<int64_t>(ne * nT * nT, 1), s);
        unsigned g2 = (unsigned)std::min<int64_t>(std::max<int64_t>(cdiv(ne * nT * nT, 256), 1), 148 * 32);
        k_scale_mats<<<g2, 256, 0, s>>>(mats, coef, ne, (int)nT, L0.AT.p);
        CK_LAUNCH();
        if (coef) {
            H.coef.alloc(std::max<int64_t>(ne, 1), s);
            CK(cudaMemcpyAsync(H.coef.p, coef, ne * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        CK(cudaStreamSynchronize(s));
    }
    trace("inputs staged");
    check_input(L0, err, s);
    trace("inputs checked");
    factor_elements(L0, err, s);
    trace("elements factored");
    build_dof_elem(L0, err, s);
    trace("dof->element map");
    L0.nnz = structural_nnz_level0(L0, err, s);
    st.stage_seconds[0] += now() - t0;
    double flops = 0.0;
    for (int l = 0;; l++) {
        Level &L = H.levels[l];
        bool last = (l == o.max_levels - 1) || L.n < o.min_coarse ||
                    (double)L.nnz / ((double)L.n * (double)L.n) > o.max_density;
        if (!last) {
            double t = now();
            trace("level %d: aggregate", l);
            aggregate_level(L, l == 0 ? o.agg_passes : o.agg_passes_coarse, err, s);
            st.stage_seconds[1] += now() - t;
            t = now();
            trace("level %d: closure (nagg %d)", l, L.nagg);
            closure_level(L, o.tau_c, o.closure, err, s);
            st.stage_seconds[2] += now() - t;
            t = now();
            trace("level %d: local spectral", l);
            g_prof_level = l;
            if (L.nagg <= 1) {
                // one aggregate: Gamma is empty and mult = 1, so S = A_ww and every mu = 1; the
                // cut keeps all modes (tau_cut < 1) or none (tau_cut >= 1) -- either way the level
                // does not coarsen and becomes the coarsest
                L.nc = (L.tau < 1.0) ? L.n : 0;
            } else {
                local_spectral(L, o, err, s, &flops);
            }
            trace("level %d: nc %lld", l, (long long)L.nc);
            st.stage_seconds[3] += now() - t;
            if (L.nc == 0 || L.nc >= L.n) last = true;  // no coarsening: this level is the coarsest
        }
        if (last) {
            double t = now();
            L.coarsest = true;
            trace("level %d: coarsest (n %lld)", l, (long long)L.n);
            { LSAMG_PROF("setup: coarsest", s); coarsest_setup(L, err, s, &flops); }
            L.AT.release();
            finish_level_info(L, s);
            st.stage_seconds[7] += now() - t;
            break;
        }
        double t = now();
        trace("level %d: colour", l);
        colour_level(L, err, s);
        trace("level %d: smoother", l);
        st.stage_seconds[4] += now() - t;
        t = now();
        {
            static const char *nm[8] = {"L0 setup: smoother factors", "L1 setup: smoother factors",
                                        "L2 setup: smoother factors", "L3 setup: smoother factors",
                                        "L4 setup: smoother factors", "L5 setup: smoother factors",
                                        "L6 setup: smoother factors", "L7 setup: smoother factors"};
            LSAMG_PROF(nm[l & 7], s);
            smoother_setup(L, o, err, s, &flops);
        }
        st.stage_seconds[5] += now() - t;
        t = now();
        H.levels.emplace_back();
        Level &Lf = H.levels[l];      // re-take references after the vector grew
        Level &Lc = H.levels[l + 1];
        trace("level %d: coarse", l);
        { LSAMG_PROF("setup: coarse gram", s); build_coarse(Lf, Lc, err, s, &flops); }
        trace("level %d: coarse built (ne %lld)", l, (long long)Lc.ne);
        Lc.nnz = structural_nnz_coarse(Lf, err, s);
        build_dof_elem(Lc, err, s);
        Lf.AT.release();
        finish_level_info(Lf, s);
        st.stage_seconds[6] += now() - t;
        if (o.verbose)
            fprintf(stderr, "[lsamg] level %d: n=%lld nagg=%d tau=%.3f ncol=%d -> n_c=%lld\n", l,
                    (long long)Lf.n, Lf.nagg, Lf.tau, Lf.ncol, (long long)Lc.n);
    }
    CK(cudaStreamSynchronize(s));
    // statistics (Section 6: level sizes, operator and grid complexity)
    st.n_levels = (int32_t)H.levels.size();
    double nnz0 = (double)H.levels[0].nnz, n0 = (double)H.levels[0].n, oc = 0, gc = 0;
    for (int l = 0; l < st.n_levels && l < 8; l++) {
        const Level &L = H.levels[l];
        st.n[l] = L.n;
        st.nnz[l] = L.nnz;
        st.n_elems[l] = L.ne;
        st.n_agg[l] = L.nagg;
        st.n_colours[l] = L.ncol;
        st.tau[l] = L.tau;
        double g = 1e300;
        for (double v : L.h_gap) g = std::min(g, v);
        st.min_gap[l] = L.coarsest ? 0.0 : g;
        oc += (double)L.nnz / nnz0;
        gc += (double)L.n / n0;
    }
    st.op_complexity = oc;
    st.grid_complexity = gc;
    st.setup_flops = flops;
    st.setup_seconds = now() - t0;
    prof_report("set-up");
}

void ensure_solve_ws(Handle &H, int nrhs) {
    cudaStream_t s = H.stream;
    for (auto &L : H.levels) ensure_cycle_ws(L, nrhs, s);
    if (H.nrhs_ws >= nrhs) return;
    int64_t n = H.n0 * nrhs;
    H.kr.alloc(n, s);
    H.kz.alloc(n, s);
    H.kp.alloc(n, s);
    H.kq.alloc(n, s);
    H.kro.alloc(n, s);
    H.kx.alloc(n, s);
    H.dots.alloc(8 * nrhs, s);
    H.nrhs_ws = nrhs;
    H.ws_gen++;   // cycle workspaces may have moved: captured V-cycles are stale
}

// One V-cycle on level 0's b -> x through a CUDA graph: captured (relaxed mode, on a private
// stream) at first use for this precision, right-hand-side count and workspace generation,
// then replayed on the handle's stream.
static void vcycle_graph(Handle &H, int nrhs, bool fp32, cudaStream_t s) {
    Handle::CycleGraph &g = H.graphs[fp32 ? 1 : 0];
    if (!g.exec || g.nrhs != nrhs || g.gen != H.ws_gen) {
        if (g.exec) {
            CK(cudaGraphExecDestroy(g.exec));
            g.exec = nullptr;
        }
        if (!H.cap_stream) CK(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(H.cap_stream, cudaStreamCaptureModeRelaxed));
        cudaGraph_t graph = nullptr;
        try {
            if (fp32)
                vcycle<float>(H, 0, nrhs, H.cap_stream);
            else
                vcycle<double>(H, 0, nrhs, H.cap_stream);
        } catch (...) {
            cudaStreamEndCapture(H.cap_stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        CK(cudaStreamEndCapture(H.cap_stream, &graph));
        const cudaError_t rc = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(rc);
        g.nrhs = nrhs;
        g.gen = H.ws_gen;
    }
    CK(cudaGraphLaunch(g.exec, s));
}

// z = B^{-1} r (one V-cycle) for FP64 vectors r, z of nrhs right-hand sides
void precondition(Handle &H, const double *r, double *z, int nrhs, bool fp32) {
    cudaStream_t s = H.stream;
    Level &L0 = H.levels[0];
    int64_t tot = L0.n * nrhs;
    // graphs only without per-kernel timing or the stage profiler (their events would be captured)
    const bool graph = H.opt.use_graph != 0 && !ktimer_enabled() && !prof_on();
    if (fp32) {
        vec_convert<double, float>(L0.b32.p, r, tot, s);
        if (graph) vcycle_graph(H, nrhs, true, s); else vcycle<float>(H, 0, nrhs, s);
        vec_convert<float, double>(z, L0.x32.p, tot, s);
    } else {
        CK(cudaMemcpyAsync(L0.b64.p, r, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (graph) vcycle_graph(H, nrhs, false, s); else vcycle<double>(H, 0, nrhs, s);
        CK(cudaMemcpyAsync(z, L0.x64.p, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
}

// Stationary V-cycle iteration x <- x + B^{-1}(b - A x) with the FP64 cycle, stopped when
// ||r_k|| <= rtol ||r_0|| (the paper's standalone solver, Section 6 preamble).
int do_stationary(Handle &H, const double *b, double *x, int nrhs, bool use_x0, int32_t *iters,
                  double *relres) {
    cudaStream_t s = H.stream;
    const lsamg_options &o = H.opt;
    ensure_solve_ws(H, nrhs);
    Level &L0 = H.levels[0];
    const int64_t n = L0.n;
    double *r = H.kr.p, *z = H.kz.p, *d = H.dots.p;
    if (!use_x0) CK(cudaMemsetAsync(x, 0, n * nrhs * sizeof(double), s));
    {
        DBuf<int> f;
        f.alloc(1, s);
        f.zero(s);
        k_nan_check<<<(unsigned)std::min<int64_t>(cdiv(n * nrhs, 256), 1184), 256, 0, s>>>(b, n * nrhs, f.p);
        CK_LAUNCH();
        if (read1(f.p, s)) fail(LSAMG_NAN, "non-finite right-hand side");
    }
    gram_spmv<double>(L0, x, r, b, nrhs, s);   // r = b - A x
    std::vector<double> r0(nrhs), rr(nrhs), hv(nrhs), step(nrhs, 1.0);
    std::vector<int32_t> its(nrhs, 0);
    std::vector<char> done(nrhs, 0);
    vec_dots(r, r, n, nrhs, d, s);
    CK(cudaMemcpyAsync(hv.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int active = 0;
    for (int i = 0; i < nrhs; i++) {
        r0[i] = std::sqrt(hv[i]);
        rr[i] = r0[i];
        done[i] = (r0[i] == 0.0);
        active += !done[i];
    }
    int it = 0;
    for (; active > 0 && it < o.maxit; it++) {
        {
            LSAMG_PROF("krylov: precondition", s);
            precondition(H, r, z, nrhs, false);
        }
        for (int i = 0; i < nrhs; i++) step[i] = done[i] ? 0.0 : 1.0;
        CK(cudaMemcpyAsync(d + 4 * nrhs, step.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        vec_axpy(x, z, d + 4 * nrhs, n, nrhs, 1.0, s);   // x += B^{-1} r (active right-hand sides)
        gram_spmv<double>(L0, x, r, b, nrhs, s);        // r = b - A x
        vec_dots(r, r, n, nrhs, d, s);
        CK(cudaMemcpyAsync(hv.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < nrhs; i++) {
            if (done[i]) continue;
            rr[i] = std::sqrt(hv[i]);
            if (!std::isfinite(rr[i])) fail(LSAMG_NAN, "non-finite residual");
            its[i] = it + 1;
            if (rr[i] <= o.rtol * r0[i]) {
                done[i] = 1;
                active--;
            }
        }
    }
    CK(cudaStreamSynchronize(s));
    for (const auto &L : H.levels) wave_check(L, s);
    prof_report("solve");
    bool ok = true;
    for (int i = 0; i < nrhs; i++) {
        if (iters) iters[i] = its[i];
        if (relres) relres[i] = r0[i] > 0.0 ? rr[i] / r0[i] : 0.0;
        ok = ok && done[i];
    }
    if (!ok) {
        g_last_error = "maximum number of iterations reached";
        return LSAMG_NO_CONVERGENCE;
    }
    return LSAMG_OK;
}

int do_solve(Handle &H, const double *b, double *x, int nrhs, int mode, bool use_x0, int32_t *iters,
             double *relres) {
    cudaStream_t s = H.stream;
    const lsamg_options &o = H.opt;
    if (mode < 0) mode = o.vcycle_fp32 ? 1 : 0;
    if (mode == 2) return do_stationary(H, b, x, nrhs, use_x0, iters, relres);
    if (mode != 0 && mode != 1) fail(LSAMG_INVALID_ARG, "solve mode must be -1, 0, 1 or 2");
    const bool fp32 = (mode == 1), flexible = (mode == 1);
    ensure_solve_ws(H, nrhs);
    Level &L0 = H.levels[0];
    const int64_t n = L0.n;
    double *r = H.kr.p, *z = H.kz.p, *p = H.kp.p, *q = H.kq.p, *ro = H.kro.p, *d = H.dots.p;
    if (!use_x0) CK(cudaMemsetAsync(x, 0, n * nrhs * sizeof(double), s));
    // r = b - A x
    gram_spmv<double>(L0, x, r, b, nrhs, s);
    {
        DBuf<int> f;
        f.alloc(1, s);
        f.zero(s);
        k_nan_check<<<(unsigned)std::min<int64_t>(cdiv(n * nrhs, 256), 1184), 256, 0, s>>>(b, n * nrhs, f.p);
        CK_LAUNCH();
        if (read1(f.p, s)) fail(LSAMG_NAN, "non-finite right-hand side");
    }
    std::vector<double> nb(nrhs), rr(nrhs), rz(nrhs), hv(3 * nrhs), alpha(nrhs), beta(nrhs);
    std::vector<int32_t> its(nrhs, 0);
    std::vector<char> done(nrhs, 0);
    vec_dots(b, b, n, nrhs, d, s);
    vec_dots(r, r, n, nrhs, d + nrhs, s);
    CK(cudaMemcpyAsync(hv.data(), d, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int active = 0;
    for (int i = 0; i < nrhs; i++) {
        nb[i] = std::sqrt(hv[i]);
        if (nb[i] == 0.0) nb[i] = 1.0;
        rr[i] = std::sqrt(hv[nrhs + i]);
        done[i] = rr[i] <= o.rtol * nb[i];
        active += !done[i];
    }
    precondition(H, r, z, nrhs, fp32);
    CK(cudaMemcpyAsync(p, z, n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    vec_dots(r, z, n, nrhs, d, s);
    CK(cudaMemcpyAsync(rz.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int it = 0;
    for (; active > 0 && it < o.maxit; it++) {
        {
            LSAMG_PROF("krylov: spmv fp64", s);
            gram_spmv<double>(L0, p, q, nullptr, nrhs, s);           // q = A p
        }
        vec_dots(p, q, n, nrhs, d, s);
        CK(cudaMemcpyAsync(hv.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < nrhs; i++) alpha[i] = (!done[i] && hv[i] != 0.0) ? rz[i] / hv[i] : 0.0;
        CK(cudaMemcpyAsync(d + 4 * nrhs, alpha.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        vec_axpy(x, p, d + 4 * nrhs, n, nrhs, 1.0, s);
        if (flexible) CK(cudaMemcpyAsync(ro, r, n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
        vec_axpy(r, q, d + 4 * nrhs, n, nrhs, -1.0, s);
        vec_dots(r, r, n, nrhs, d, s);
        CK(cudaMemcpyAsync(hv.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < nrhs; i++) {
            if (done[i]) continue;
            rr[i] = std::sqrt(hv[i]);
            if (!std::isfinite(rr[i])) fail(LSAMG_NAN, "non-finite residual");
            its[i] = it + 1;
            if (rr[i] <= o.rtol * nb[i]) {
                done[i] = 1;
                active--;
            }
        }
        if (active == 0) {
            it++;
            break;
        }
        {
            LSAMG_PROF("krylov: precondition", s);
            precondition(H, r, z, nrhs, fp32);
        }
        vec_dots(r, z, n, nrhs, d, s);
        if (flexible) vec_dots(ro, z, n, nrhs, d + nrhs, s);
        CK(cudaMemcpyAsync(hv.data(), d, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < nrhs; i++) {
            double rzn = hv[i];
            double bt;
            if (flexible)  // Polak-Ribiere: z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k)
                bt = (rzn - hv[nrhs + i]) / rz[i];
            else
                bt = rzn / rz[i];
            beta[i] = done[i] ? 0.0 : bt;
            rz[i] = rzn;
        }
        CK(cudaMemcpyAsync(d + 5 * nrhs, beta.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        vec_xpby(p, z, d + 5 * nrhs, n, nrhs, s);
    }
    CK(cudaStreamSynchronize(s));
    for (const auto &L : H.levels) wave_check(L, s);
    prof_report("solve");
    bool ok = true;
    for (int i = 0; i < nrhs; i++) {
        if (iters) iters[i] = done[i] ? its[i] : it;
        if (relres) relres[i] = rr[i] / nb[i];
        ok = ok && done[i];
    }
    if (!ok) {
        g_last_error = "maximum number of iterations reached";
        return LSAMG_NO_CONVERGENCE;
    }
    return LSAMG_OK;
}

}  // namespace
}  // namespace lsamg

using namespace lsamg;

struct lsamg_handle {
    Handle h;
};

static void set_sweep_globals(const lsamg_options &o) {
    g_split_sweep = o.split_sweep > 0 ? o.split_sweep : 128;
    g_sweep_block = o.sweep_block > 0 ? std::min(o.sweep_block, 64) : 64;
}

extern "C" {

lsamg_options lsamg_options_default(void) {
    lsamg_options o;
    memset(&o, 0, sizeof o);
    o.tau_c = 0.75;
    o.agg_passes = 2;
    o.agg_passes_coarse = 2;
    o.max_levels = 3;
    o.min_coarse = 10;
    o.max_density = 0.25;
    o.vcycle_fp32 = 1;
    o.maxit = 1000;
    o.rtol = 1e-8;
    o.chunk_bytes = 0;
    o.use_graph = 0;
    o.verbose = 0;
    o.profile = 0;
    o.large_dense = 0;
    o.split_sweep = 0;
    o.sweep_block = 0;
    o.smoother = 0;
    o.closure = 0;
    return o;
}

int32_t lsamg_kernel_classes(void) { return KC_N; }
const char *lsamg_kernel_name(int32_t cls) { return kclass_name(cls); }
int lsamg_kernel_stats_all(double *out) {
    if (!out) return LSAMG_INVALID_ARG;
    return guarded([&] {
        KStat st[KC_N];
        ktimer_collect(st);
        for (int c = 0; c < KC_N; c++) {
            out[4 * c + 0] = st[c].ms;
            out[4 * c + 1] = (double)st[c].calls;
            out[4 * c + 2] = st[c].flops;
            out[4 * c + 3] = st[c].bytes;
        }
    });
}
int64_t lsamg_launch_count(void) { return launch_count(); }

int lsamg_setup(const lsamg_problem *prob, const lsamg_options *opts, void *stream,
                lsamg_handle **out) {
    if (!out) return LSAMG_INVALID_ARG;
    *out = nullptr;
    lsamg_handle *h = new (std::nothrow) lsamg_handle();
    if (!h) return LSAMG_OOM;
    h->h.stream = (cudaStream_t)stream;
    h->h.opt = opts ? *opts : lsamg_options_default();
    ktimer_enable(h->h.opt.profile != 0);
    g_large_dense = h->h.opt.large_dense > 0 ? h->h.opt.large_dense : 2048;
    set_sweep_globals(h->h.opt);
    int rc = guarded([&] { do_setup(h->h, prob, h->h.opt); });
    if (rc != LSAMG_OK) {
        std::string msg = g_last_error;
        cudaStreamSynchronize(h->h.stream);
        delete h;
        g_last_error = msg;
        return rc;
    }
    *out = h;
    return LSAMG_OK;
}

int lsamg_apply(lsamg_handle *h, const double *r, double *z, int32_t nrhs, int32_t fp32,
                void *stream) {
    if (!h || !r || !z || nrhs < 1) return LSAMG_INVALID_ARG;
    return guarded([&] {
        Handle &H = h->h;
        H.stream = (cudaStream_t)stream;
        set_sweep_globals(H.opt);
        ensure_solve_ws(H, nrhs);
        bool f = fp32 < 0 ? H.opt.vcycle_fp32 != 0 : fp32 != 0;
        precondition(H, r, z, nrhs, f);
        CK(cudaStreamSynchronize(H.stream));
        for (const auto &L : H.levels) wave_check(L, H.stream);
    });
}

int lsamg_solve(lsamg_handle *h, const double *b, double *x, int32_t nrhs, int32_t mode,
                int32_t use_x0, void *stream, int32_t *iters, double *relres) {
    if (!h || !b || !x || nrhs < 1) return LSAMG_INVALID_ARG;
    int status = LSAMG_OK;
    int rc = guarded([&] {
        Handle &H = h->h;
        H.stream = (cudaStream_t)stream;
        set_sweep_globals(H.opt);
        status = do_solve(H, b, x, nrhs, mode, use_x0 != 0, iters, relres);
    });
    if (rc != LSAMG_OK) return rc;
    return status;
}

int lsamg_solve_host(lsamg_handle *h, const double *b_host, double *x_host, int32_t nrhs,
                     int32_t mode, void *stream, int32_t *iters, double *relres) {
    if (!h || !b_host || !x_host || nrhs < 1) return LSAMG_INVALID_ARG;
    int status = LSAMG_OK;
    int rc = guarded([&] {
        Handle &H = h->h;
        H.stream = (cudaStream_t)stream;
        int64_t cnt = H.n0 * nrhs;
        DBuf<double> db, dx;
        db.alloc(cnt, H.stream);
        dx.alloc(cnt, H.stream);
        CK(cudaMemcpyAsync(db.p, b_host, cnt * sizeof(double), cudaMemcpyHostToDevice, H.stream));
        status = do_solve(H, db.p, dx.p, nrhs, mode, false, iters, relres);
        CK(cudaMemcpyAsync(x_host, dx.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
        CK(cudaStreamSynchronize(H.stream));
    });
    if (rc != LSAMG_OK) return rc;
    return status;
}

int lsamg_gram_spmv(lsamg_handle *h, int32_t level, const void *x, void *y, int32_t fp32,
                    void *stream) {
    if (!h || !x || !y || level < 0 || level >= (int)h->h.levels.size()) return LSAMG_INVALID_ARG;
    return guarded([&] {
        Handle &H = h->h;
        cudaStream_t s = (cudaStream_t)stream;
        const Level &L = H.levels[level];
        if (fp32)
            gram_spmv<float>(L, (const float *)x, (float *)y, nullptr, 1, s);
        else
            gram_spmv<double>(L, (const double *)x, (double *)y, nullptr, 1, s);
        CK(cudaStreamSynchronize(s));
    });
}

int lsamg_dgemm_nt(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda, const double *B,
                   int64_t ldb, double beta, double *C, int64_t ldc, void *stream) {
    if (M < 0 || N < 0 || K < 0 || (M > 0 && lda < M) || (N > 0 && ldb < N) || (M > 0 && ldc < M))
        return LSAMG_INVALID_ARG;
    if (M > 0x7fffffff || N > 0x7fffffff || K > 0x7fffffff) return LSAMG_LIMIT;
    if (M == 0 || N == 0) return LSAMG_OK;
    if (!A || !B || !C) return LSAMG_INVALID_ARG;
    return guarded([&] {
        cudaStream_t s = (cudaStream_t)stream;
        DBuf<int> err;
        err.alloc(2, s);
        err.zero(s);
        oz::Workspace ws;
        if (K == 0) {   // C = beta C through a product with a zero operand
            DBuf<double> z;
            z.alloc(1, s);
            z.zero(s);
            std::vector<oz::SplitJob> sj{{0, 0, 0, 0, 0, (int32_t)M, 1}, {0, 0, 0, 0, 0, (int32_t)N, 1}};
            sj[1].dst_off = oz::slice_halves(M, 1);
            sj[1].exp_off = oz::exp_ints(M);
            ws.reserve(sj[1].dst_off + oz::slice_halves(N, 1), sj[1].exp_off + oz::exp_ints(N), s);
            oz::split(z.p, sj, ws.sl.p, ws.ex.p, s);
            oz::gemm(ws.sl.p, ws.ex.p, C, {oz::GemmJob{0, sj[1].dst_off, 0, sj[1].exp_off, 0, 1, ldc, (int32_t)M,
                                                     (int32_t)N, 1, 0, 0, 0}},
                     0.0, beta, err.p, s);
        } else {
            // the products run in K passes of at most 4096 (oz::gemm), the operands are split once
            const int64_t hb = oz::slice_halves(M, K), eb = oz::exp_ints(M);
            std::vector<oz::SplitJob> sa{{0, 1, lda, 0, 0, (int32_t)M, (int32_t)K}};
            std::vector<oz::SplitJob> sb{{0, 1, ldb, hb, eb, (int32_t)N, (int32_t)K}};
            ws.reserve(hb + oz::slice_halves(N, K), eb + oz::exp_ints(N), s);
            oz::split(A, sa, ws.sl.p, ws.ex.p, s);
            oz::split(B, sb, ws.sl.p, ws.ex.p, s);
            oz::gemm(ws.sl.p, ws.ex.p, C,
                     {oz::GemmJob{0, hb, 0, eb, 0, 1, ldc, (int32_t)M, (int32_t)N, (int32_t)K, 0, 0, 0}}, alpha, beta,
                     err.p, s);
        }
        check_err(err.p, s, "tensor-core FP64 product");
    });
}

int lsamg_elem_grad(lsamg_handle *h, const double *lam, const double *x, double *g, void *stream) {
    if (!h || !lam || !x || !g) return LSAMG_INVALID_ARG;
    if (!h->h.coef.p) {
        g_last_error = "element coefficients were not given at set-up";
        return LSAMG_INVALID_ARG;
    }
    return guarded([&] {
        cudaStream_t s = (cudaStream_t)stream;
        elem_grad(h->h.levels[0], h->h.coef.p, lam, x, g, s);
        CK(cudaStreamSynchronize(s));
    });
}

int lsamg_get_stats(lsamg_handle *h, lsamg_stats *out) {
    if (!h || !out) return LSAMG_INVALID_ARG;
    *out = h->h.stats;
    return LSAMG_OK;
}

const char *lsamg_stage_name(int32_t i) {
    if (i < 0 || i >= (int32_t)(sizeof(kStages) / sizeof(kStages[0]))) return "";
    return kStages[i];
}

int lsamg_query(lsamg_handle *h, int32_t level, int32_t what, void *out, int64_t cap_bytes,
                int64_t *bytes_needed) {
    if (!h || level < 0 || level >= (int)h->h.levels.size()) return LSAMG_INVALID_ARG;
    return guarded([&] {
        Handle &H = h->h;
        Level &L = H.levels[level];
        const void *src = nullptr;
        int64_t bytes = 0;
        auto pick = [&](const void *p, int64_t b) {
            src = p;
            bytes = b;
        };
        switch (what) {
            case LSAMG_Q_AGG: pick(L.agg.p, L.agg.p ? L.n * 4 : 0); break;
            case LSAMG_Q_MULT: pick(L.mult.p, L.mult.p ? L.ne * 4 : 0); break;
            case LSAMG_Q_OMEGA_PTR: pick(L.Optr.p, L.Optr.p ? (L.nagg + 1) * 8 : 0); break;
            case LSAMG_Q_OMEGA_IDX: pick(L.Oidx.p, L.Optr.p ? L.Omega_total * 4 : 0); break;
            case LSAMG_Q_K: pick(L.k.p, L.k.p ? (int64_t)L.nagg * 4 : 0); break;
            case LSAMG_Q_ZOFF: pick(L.zoff.p, L.zoff.p ? (L.nagg + 1) * 8 : 0); break;
            case LSAMG_Q_Z:
                pick(L.Z64.p, L.zoff.p ? read1(L.zoff.p + L.nagg, H.stream) * 8 : 0);
                break;
            case LSAMG_Q_CELEM_PTR:
                if (level + 1 < (int)H.levels.size())
                    pick(H.levels[level + 1].eptr.p, (H.levels[level + 1].ne + 1) * 8);
                break;
            case LSAMG_Q_CELEM_IDX:
                if (level + 1 < (int)H.levels.size())
                    pick(H.levels[level + 1].eidx.p, H.levels[level + 1].nnz_e * 4);
                break;
            case LSAMG_Q_GOFF: pick(L.goff.p, (L.ne + 1) * 8); break;
            case LSAMG_Q_GROWS: pick(L.grows.p, L.ne * 4); break;
            case LSAMG_Q_G: pick(L.G64.p, L.G64.n * 8); break;
            case LSAMG_Q_COLOUR: pick(L.colour.p, L.colour.p ? (int64_t)L.nagg * 4 : 0); break;
            case LSAMG_Q_EPTR: pick(L.eptr.p, (L.ne + 1) * 8); break;
            case LSAMG_Q_EIDX: pick(L.eidx.p, L.nnz_e * 4); break;
            case LSAMG_Q_MU:
                if (bytes_needed) *bytes_needed = (int64_t)L.h_gap.size() * 8;
                if (out && cap_bytes >= (int64_t)L.h_gap.size() * 8 && !L.h_gap.empty())
                    memcpy(out, L.h_gap.data(), L.h_gap.size() * 8);
                return;
            case LSAMG_Q_CGROUP: pick(L.cgroup.p, L.cgroup.p ? L.ne * 4 : 0); break;
            default: fail(LSAMG_INVALID_ARG, "unknown query");
        }
        if (bytes_needed) *bytes_needed = bytes;
        if (out && src && bytes > 0 && cap_bytes >= bytes) {
            CK(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, H.stream));
            CK(cudaStreamSynchronize(H.stream));
        }
    });
}

void lsamg_destroy(lsamg_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->h.stream);
    delete h;
    cudaDeviceSynchronize();
}

const char *lsamg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
