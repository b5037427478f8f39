// C ABI of libtdarisp (declared in include/tdarisp.h).  Every entry point
// converts internal exceptions into a status code and keeps the message in
// the context.
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "ctx.cuh"
#include "linalg.cuh"

namespace {

template <typename F>
int guarded(tr_ctx *c, F &&f)
{
    if (!c) return TR_EINVAL;
    try {
        c->err.clear();
        return f();
    } catch (const tr::Error &e) {
        c->err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        c->err = e.what();
        return TR_ECUDA;
    }
}

void fill_defaults(tr_options *o)
{
    std::memset(o, 0, sizeof *o);
    o->cx = 0.25;
    o->k_alpha = 1.0;
    o->k_beta = 0.0;
    o->omega = 0.0;
    o->window_ev = 40.0;
    o->aux_on_h = 0;
    o->nstates = 5;
    o->block = 0;
    o->max_space = 0;
    o->max_iter = 0;
    o->tol = 1e-5;
    o->precision = TR_FP64;
    o->screen = 1e-22;
    o->hbm_budget = 0;
    o->aux_chunk_bytes = 0;
}

void normalise_options(tr_options *o)
{
    if (!(o->screen > 0.0)) o->screen = 1e-22;
    if (o->aux_chunk_bytes == 0) o->aux_chunk_bytes = (size_t)12 << 30;
    if (o->matvec_ws_bytes == 0) o->matvec_ws_bytes = (size_t)4 << 30;
}

// the bounded waits of the context's tensor-core launches follow its options
void apply_wait_options(tr_ctx *c)
{
    TR_REQUIRE(c->opt.wait_cycles >= 0, TR_EINVAL, "options: wait_cycles must be >= 0");
    TR_REQUIRE(c->opt.wait_test == 0 || c->opt.wait_test == 1, TR_EINVAL, "options: wait_test must be 0 or 1");
    c->prof.wait_cycles = c->opt.wait_cycles;
    c->prof.wait_stall = c->opt.wait_test;
}

}  // namespace

extern "C" {

int tr_version(void) { return 100; }

void tr_options_default(tr_options *opt)
{
    if (opt) fill_defaults(opt);
}

int tr_create(tr_ctx **out, const tr_options *opt, void *cuda_stream)
{
    if (!out || !opt) return TR_EINVAL;
    *out = nullptr;
    tr_ctx *c = nullptr;
    try {
        c = new tr_ctx();
    } catch (...) {
        return TR_ENOMEM;
    }
    int rc = guarded(c, [&]() {
        TR_REQUIRE(opt->precision == TR_FP64 || opt->precision == TR_MIXED || opt->precision == TR_FP64_TC,
                   TR_EINVAL, "create: precision must be TR_FP64, TR_MIXED or TR_FP64_TC");
        TR_REQUIRE(opt->xform_slices == 0 || opt->xform_slices == -1 ||
                       (opt->xform_slices >= 2 && opt->xform_slices <= 7),
                   TR_EINVAL, "create: xform_slices must be -1, 0 or 2..7");
        TR_REQUIRE(opt->j_ao == 0 || opt->j_ao == 1, TR_EINVAL, "create: j_ao must be 0 or 1");
        TR_REQUIRE(opt->tddft == 0 || opt->tddft == 1, TR_EINVAL, "create: tddft must be 0 or 1");
        TR_REQUIRE(!opt->tddft || opt->precision != TR_MIXED, TR_EINVAL,
                   "create: full TDDFT (tddft = 1) needs precision TR_FP64 or TR_FP64_TC");
        c->opt = *opt;
        normalise_options(&c->opt);
        apply_wait_options(c);
        c->st = (cudaStream_t)cuda_stream;
        TR_CUDA(cudaGetDevice(&c->device));
        tr::gemm_prepare();
        size_t fr = 0, tot = 0;
        TR_CUDA(cudaMemGetInfo(&fr, &tot));
        c->budget.limit = opt->hbm_budget ? opt->hbm_budget : (size_t)(0.9 * (double)fr);
        return TR_OK;
    });
    if (rc != TR_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return TR_OK;
}

void tr_destroy(tr_ctx *ctx) { delete ctx; }

const char *tr_last_error(const tr_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tr_set_options(tr_ctx *ctx, const tr_options *opt)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(opt, TR_EINVAL, "set_options: null options");
        TR_REQUIRE(opt->precision == TR_FP64 || opt->precision == TR_MIXED || opt->precision == TR_FP64_TC,
                   TR_EINVAL, "set_options: precision must be TR_FP64, TR_MIXED or TR_FP64_TC");
        TR_REQUIRE(opt->xform_slices == 0 || opt->xform_slices == -1 ||
                       (opt->xform_slices >= 2 && opt->xform_slices <= 7),
                   TR_EINVAL, "set_options: xform_slices must be -1, 0 or 2..7");
        TR_REQUIRE(opt->j_ao == 0 || opt->j_ao == 1, TR_EINVAL, "set_options: j_ao must be 0 or 1");
        TR_REQUIRE(opt->tddft == 0 || opt->tddft == 1, TR_EINVAL, "set_options: tddft must be 0 or 1");
        TR_REQUIRE(!opt->tddft || opt->precision != TR_MIXED, TR_EINVAL,
                   "set_options: full TDDFT (tddft = 1) needs precision TR_FP64 or TR_FP64_TC");
        bool rebuild = opt->precision != ctx->opt.precision || opt->cx != ctx->opt.cx || opt->k_alpha != ctx->opt.k_alpha ||
                       opt->k_beta != ctx->opt.k_beta || opt->omega != ctx->opt.omega ||
                       opt->window_ev != ctx->opt.window_ev || opt->aux_on_h != ctx->opt.aux_on_h ||
                       opt->screen != ctx->opt.screen || opt->xform_slices != ctx->opt.xform_slices ||
                       opt->j_ao != ctx->opt.j_ao || opt->tddft != ctx->opt.tddft;
        TR_REQUIRE(opt->wait_cycles >= 0 && (opt->wait_test == 0 || opt->wait_test == 1), TR_EINVAL,
                   "set_options: wait_cycles must be >= 0 and wait_test 0 or 1");
        size_t limit = ctx->budget.limit;
        ctx->opt = *opt;
        normalise_options(&ctx->opt);
        apply_wait_options(ctx);
        if (opt->hbm_budget) ctx->budget.limit = opt->hbm_budget;
        else ctx->budget.limit = limit;
        if (rebuild) {
            ctx->built = false;
            if (ctx->have_mol) tr::refresh_molecule(ctx);
            if (ctx->have_orb) tr::refresh_window(ctx);
        }
        return TR_OK;
    });
}

int tr_set_molecule(tr_ctx *ctx, int natm, const int *Z, const double *xyz, const double *aux_exp,
                    int nshell, const tr_shell *shells)
{
    return guarded(ctx, [&]() {
        tr::set_molecule(ctx, natm, Z, xyz, aux_exp, nshell, shells);
        return TR_OK;
    });
}

int tr_set_orbitals(tr_ctx *ctx, int nao, int nmo, int nocc, const double *C, const double *eps, int on_device)
{
    return guarded(ctx, [&]() {
        tr::set_orbitals(ctx, nao, nmo, nocc, C, eps, on_device);
        return TR_OK;
    });
}

int tr_get_dims(tr_ctx *ctx, tr_dims *out)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(out, TR_EINVAL, "get_dims: null output");
        std::memset(out, 0, sizeof *out);
        out->nao = ctx->nao;
        out->nmo = ctx->nmo;
        out->nocc = ctx->nocc;
        out->nvir = ctx->nvir;
        out->naux_j = ctx->nJ;
        out->naux_k = ctx->nK;
        out->occ_k0 = ctx->o0;
        out->nocc_k = ctx->oK;
        out->nvir_k = ctx->vK;
        out->npair = (int)ctx->pl.pairs.size();
        out->ntotal_pair = ctx->pl.ntotal;
        return TR_OK;
    });
}

int tr_build(tr_ctx *ctx)
{
    return guarded(ctx, [&]() {
        tr::build(ctx);
        return TR_OK;
    });
}

int tr_int3c(tr_ctx *ctx, int which, int p0, int np, double *out_dev)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(out_dev || np == 0, TR_EINVAL, "int3c: null output");
        tr::int3c_ao(ctx, which, p0, np, out_dev);
        return TR_OK;
    });
}

int tr_int2c(tr_ctx *ctx, int which, double *out_dev)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(out_dev, TR_EINVAL, "int2c: null output");
        tr::int2c_aux(ctx, which, out_dev);
        return TR_OK;
    });
}

int tr_get_tensor(tr_ctx *ctx, int which, double *out, int on_device)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(out, TR_EINVAL, "get_tensor: null output");
        tr::get_tensor(ctx, which, out, on_device);
        return TR_OK;
    });
}

int tr_transition_dipoles(tr_ctx *ctx, int n, const double *X, const double *origin, double *mu, int on_device)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(n >= 0, TR_EINVAL, "transition_dipoles: n must be >= 0");
        if (n == 0) return TR_OK;
        TR_REQUIRE(X && mu, TR_EINVAL, "transition_dipoles: null pointer");
        const double O[3] = {origin ? origin[0] : 0.0, origin ? origin[1] : 0.0, origin ? origin[2] : 0.0};
        const size_t nx = (size_t)n * ctx->nov;
        tr::DevBuf<double> xd, md;
        const double *Xd = X;
        double *mud = mu;
        if (!on_device) {
            xd.alloc(nx, &ctx->budget, "excitation vectors");
            md.alloc((size_t)3 * n, &ctx->budget, "transition dipoles");
            TR_CUDA(cudaMemcpyAsync(xd.p, X, sizeof(double) * nx, cudaMemcpyHostToDevice, ctx->st));
            Xd = xd.p;
            mud = md.p;
        }
        tr::transition_dipoles(ctx, n, Xd, O, mud);
        if (!on_device) {
            TR_CUDA(cudaMemcpyAsync(mu, md.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->st));
            TR_CUDA(cudaStreamSynchronize(ctx->st));
        }
        return TR_OK;
    });
}

int tr_oscillator_strengths(tr_ctx *ctx, int n, const double *omega, const double *X, double *f, int on_device)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(n >= 0, TR_EINVAL, "oscillator_strengths: n must be >= 0");
        if (n == 0) return TR_OK;
        TR_REQUIRE(omega && X && f, TR_EINVAL, "oscillator_strengths: null pointer");
        const size_t nx = (size_t)n * ctx->nov;
        tr::DevBuf<double> xd, od, fd;
        const double *Xd = X, *Od = omega;
        double *Fd = f;
        if (!on_device) {
            xd.alloc(nx, &ctx->budget, "excitation vectors");
            od.alloc(n, &ctx->budget, "excitation energies");
            fd.alloc(n, &ctx->budget, "oscillator strengths");
            TR_CUDA(cudaMemcpyAsync(xd.p, X, sizeof(double) * nx, cudaMemcpyHostToDevice, ctx->st));
            TR_CUDA(cudaMemcpyAsync(od.p, omega, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
            Xd = xd.p;
            Od = od.p;
            Fd = fd.p;
        }
        tr::oscillator_strengths(ctx, n, Od, Xd, Fd);
        if (!on_device) {
            TR_CUDA(cudaMemcpyAsync(f, fd.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st));
            TR_CUDA(cudaStreamSynchronize(ctx->st));
        }
        return TR_OK;
    });
}

int tr_matvec(tr_ctx *ctx, int m, const double *X, double *AX, int on_device)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(m >= 0, TR_EINVAL, "matvec: m must be >= 0");
        TR_REQUIRE(ctx->built, TR_EINVAL, "matvec: call tr_build first");
        if (m == 0) return TR_OK;
        TR_REQUIRE(X && AX, TR_EINVAL, "matvec: null pointer");
        const size_t n = (size_t)m * ctx->nov;
        if (on_device) {
            TR_REQUIRE(X + n <= AX || AX + n <= X, TR_EINVAL, "matvec: X and AX overlap");
            tr::matvec(ctx, m, X, AX);
            return TR_OK;
        }
        tr::DevBuf<double> dx, dax;
        dx.alloc(n, &ctx->budget, "matvec input");
        dax.alloc(n, &ctx->budget, "matvec output");
        TR_CUDA(cudaMemcpyAsync(dx.p, X, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
        TR_CUDA(cudaMemsetAsync(ctx->flag.p + 1, 0, sizeof(int), ctx->st));
        tr::matvec(ctx, m, dx.p, dax.p);
        TR_CUDA(cudaMemcpyAsync(AX, dax.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st));
        int tc_err = 0;
        TR_CUDA(cudaMemcpyAsync(&tc_err, ctx->flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        TR_CUDA(cudaStreamSynchronize(ctx->st));
        TR_REQUIRE(!tc_err, TR_ETIMEOUT,
                   "matvec: a tensor-core pipeline wait ran out (code " + std::to_string(tc_err) + ")");
        return TR_OK;
    });
}

int tr_solve(tr_ctx *ctx, double *omega, double *X, double *resid, int on_device, tr_solve_info *info)
{
    return guarded(ctx, [&]() { return tr::solve(ctx, omega, X, nullptr, resid, on_device, info); });
}

int tr_solve_tddft(tr_ctx *ctx, double *omega, double *XpY, double *XmY, double *resid, int on_device,
                   tr_solve_info *info)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(ctx->opt.tddft, TR_EINVAL, "solve_tddft: the context was not set up with tddft = 1");
        return tr::solve(ctx, omega, XpY, XmY, resid, on_device, info);
    });
}

int tr_matvec_tddft(tr_ctx *ctx, int m, const double *X, double *ApBX, double *AmBX, int on_device)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(m >= 0, TR_EINVAL, "matvec_tddft: m must be >= 0");
        TR_REQUIRE(ctx->opt.tddft, TR_EINVAL, "matvec_tddft: the context was not set up with tddft = 1");
        TR_REQUIRE(ctx->built, TR_EINVAL, "matvec_tddft: call tr_build first");
        if (m == 0) return TR_OK;
        TR_REQUIRE(X && ApBX && AmBX, TR_EINVAL, "matvec_tddft: null pointer");
        const size_t n = (size_t)m * ctx->nov;
        if (on_device) {
            auto apart = [n](const double *a, const double *b) { return a + n <= b || b + n <= a; };
            TR_REQUIRE(apart(X, ApBX) && apart(X, AmBX) && apart(ApBX, AmBX), TR_EINVAL,
                       "matvec_tddft: X, ApBX and AmBX overlap");
            tr::matvec_pm(ctx, m, X, ApBX, AmBX);
            return TR_OK;
        }
        tr::DevBuf<double> dx, dp, dm;
        dx.alloc(n, &ctx->budget, "matvec input");
        dp.alloc(n, &ctx->budget, "matvec output");
        dm.alloc(n, &ctx->budget, "matvec output");
        TR_CUDA(cudaMemcpyAsync(dx.p, X, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
        TR_CUDA(cudaMemsetAsync(ctx->flag.p + 1, 0, sizeof(int), ctx->st));
        tr::matvec_pm(ctx, m, dx.p, dp.p, dm.p);
        TR_CUDA(cudaMemcpyAsync(ApBX, dp.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st));
        TR_CUDA(cudaMemcpyAsync(AmBX, dm.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st));
        int tc_err = 0;
        TR_CUDA(cudaMemcpyAsync(&tc_err, ctx->flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        TR_CUDA(cudaStreamSynchronize(ctx->st));
        TR_REQUIRE(!tc_err, TR_ETIMEOUT,
                   "matvec_tddft: a tensor-core pipeline wait ran out (code " + std::to_string(tc_err) + ")");
        return TR_OK;
    });
}

int tr_build_batch(tr_ctx **ctxs, int n, int nthreads)
{
    if (!ctxs || n <= 0) return TR_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return TR_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TR_ECUDA;
    if (nthreads <= 0) nthreads = 8;
    nthreads = std::min(nthreads, n);
    // every context builds on a stream of its own
    std::vector<cudaStream_t> orig(n), own(n, nullptr);
    for (int i = 0; i < n; ++i) {
        orig[i] = ctxs[i]->st;
        if (cudaStreamSynchronize(orig[i]) != cudaSuccess || cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking) != cudaSuccess) {
            for (int j = 0; j < i; ++j) {
                ctxs[j]->st = orig[j];
                cudaStreamDestroy(own[j]);
            }
            return TR_ECUDA;
        }
        ctxs[i]->st = own[i];
    }
    std::vector<int> rc(n, TR_OK);
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    // the build temporaries of each context go back to its block pool rather
    // than to cudaFree (which waits for the whole device, so concurrent builds
    // would serialise on each other's frees), and its next batched build takes
    // them again
    for (int i = 0; i < n; ++i) ctxs[i]->budget.pool.on = true;
    for (int t = 0; t < nthreads; ++t)
        pool.emplace_back([&]() {
            cudaSetDevice(dev);
            for (int i = next++; i < n; i = next++) rc[i] = tr_build(ctxs[i]);
        });
    for (auto &t : pool) t.join();
    int out = TR_OK;
    for (int i = 0; i < n; ++i) {
        cudaStreamSynchronize(own[i]);
        ctxs[i]->budget.pool.on = false;
        ctxs[i]->st = orig[i];
        cudaStreamDestroy(own[i]);
        if (rc[i] != TR_OK && out == TR_OK) out = rc[i];
    }
    return out;
}

int tr_solve_batch(tr_ctx **ctxs, int n, double **omega, double **X, double **resid, int on_device,
                   tr_solve_info *infos, int autotune_tiles)
{
    if (!ctxs || n <= 0 || !ctxs[0]) return TR_EINVAL;
    tr_ctx *c0 = ctxs[0];
    int rc = guarded(c0, [&]() {
        for (int i = 0; i < n; ++i) TR_REQUIRE(ctxs[i], TR_EINVAL, "solve_batch: null context");
        return tr::solve_batch(ctxs, n, omega, X, resid, on_device, infos, autotune_tiles);
    });
    for (int i = 1; i < n; ++i)
        if (ctxs[i]) ctxs[i]->err = c0->err;
    return rc;
}

int tr_profile(tr_ctx *ctx, int enable)
{
    return guarded(ctx, [&]() {
        ctx->prof.reset();
        ctx->prof.enabled = enable != 0;
        return TR_OK;
    });
}

int tr_profile_get(tr_ctx *ctx, tr_prof_entry *out, int max)
{
    return guarded(ctx, [&]() {
        ctx->prof.flush();
        int n = (int)ctx->prof.names.size();
        for (int i = 0; i < n && i < max && out; ++i) {
            std::memset(&out[i], 0, sizeof out[i]);
            std::strncpy(out[i].name, ctx->prof.names[i].c_str(), sizeof(out[i].name) - 1);
            out[i].launches = ctx->prof.n[i];
            out[i].total_ms = ctx->prof.ms[i];
            out[i].flops = ctx->prof.fl[i];
            out[i].bytes = ctx->prof.by[i];
        }
        return n;
    });
}

long tr_launch_count(const tr_ctx *ctx) { return ctx ? ctx->prof.launches : 0; }

int tr_subspace_eigh(tr_ctx *ctx, int k, const double *H, int nev, double *w, double *Y, int on_device)
{
    return guarded(ctx, [&]() {
        TR_REQUIRE(k > 0 && nev > 0 && nev <= k && H && w && Y, TR_EINVAL, "subspace_eigh: bad arguments");
        tr::DevBuf<double> A, sw, sY, scr;
        A.alloc((size_t)k * k, &ctx->budget, "eigh matrix");
        sw.alloc(nev, &ctx->budget, "eigh values");
        sY.alloc((size_t)k * nev, &ctx->budget, "eigh vectors");
        scr.alloc(tr::eigh_lowest_scratch(k, nev) / sizeof(double), &ctx->budget, "eigh scratch");
        if (!ctx->flag.p) ctx->flag.alloc(4, &ctx->budget, "flags");
        const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const cudaMemcpyKind out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        TR_CUDA(cudaMemcpyAsync(A.p, H, sizeof(double) * (size_t)k * k, in, ctx->st));
        tr::eigh_lowest(ctx->prof, ctx->st, A.p, k, nev, sw.p, sY.p, nev, scr.p, ctx->flag.p);
        TR_CUDA(cudaGetLastError());
        TR_CUDA(cudaMemcpyAsync(w, sw.p, sizeof(double) * nev, out, ctx->st));
        TR_CUDA(cudaMemcpyAsync(Y, sY.p, sizeof(double) * (size_t)k * nev, out, ctx->st));
        TR_CUDA(cudaStreamSynchronize(ctx->st));
        return TR_OK;
    });
}

int tr_memory(tr_ctx *ctx, size_t *used, size_t *peak, size_t *estimate)
{
    return guarded(ctx, [&]() {
        if (used) *used = ctx->budget.used;
        if (peak) *peak = ctx->budget.peak;
        if (estimate) {
            TR_REQUIRE(ctx->have_mol && ctx->have_orb, TR_EINVAL, "memory: molecule and orbitals required");
            *estimate = tr::footprint(ctx);
        }
        return TR_OK;
    });
}

}  // extern "C"
