// Several independent problems in one call: the k-points and spin channels of a periodic
// calculation (arXiv:1705.11191 sec. 2, SINGLE_PROC mode: one process solves a group of
// k-points one after another), with the chemical potential shared across them (sec. 4.4:
// the electron count of the bisection is summed over k-points, spin channels and states).
//
// Three phases, each also exported on its own so that several processes can split the
// problems between them and exchange only the eigenvalues (elsi_gb.h):
//   1. batch_ev: eigenpairs of each problem, kept in the handle (real form for complex
//      problems: vectors of length 2n, two per complex state);
//   2. occupation: one chemical potential over all kept eigenvalues with the problems'
//      weights (occupation_weighted), or one per problem;
//   3. batch_dm: P_i = C_i diag(f_i) C_i^H and W_i = C_i diag(f_i eps_i) C_i^H, and the
//      band energy sum_l f_il eps_il of each problem.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

struct BatchItem {
    int n = 0, k = 0;        // basis size, number of states (complex count for complex problems)
    size_t off_val = 0;      // real-form eigenvalues: N = n or 2n entries
    size_t off_vec = 0;      // real-form eigenvectors: N x K, K = k or 2k
    size_t off_lvl = 0;      // state eigenvalues / occupations: k entries
};

struct BatchWorker {
    elsi_gb_handle_s *sub = nullptr;  // solver instance of this worker
    cudaStream_t stream = nullptr;    // its stream (created here)
};

struct BatchState {
    elsi_gb_handle_s *sub = nullptr;  // solver instance the problems run in (worker 0)
    std::vector<BatchWorker> workers; // workers 1 .. W-1 (own handle, stream, host thread)
    std::vector<BatchItem> items;
    bool cplx = false;
    size_t total_lvl = 0;
#define EGB_BUF(type, name) type *name = nullptr; size_t name##_cap = 0;
    EGB_BUF(double, vals)
    EGB_BUF(double, vecs)
    EGB_BUF(double, lvl)    // eigenvalue of each state (concatenated over problems)
    EGB_BUF(double, wts)    // weight of each state
    EGB_BUF(double, occ)    // occupation of each state
    EGB_BUF(double, occ2)   // complex problems: occupations duplicated over the pairs
    EGB_BUF(double, emb)    // complex problems: P, W of the real form (2n x 2n each)
    EGB_BUF(double, cw)     // density scratch (N x K)
    EGB_BUF(double, outs)   // per-problem scalars
    EGB_BUF(int, offs)      // state offsets (nprob + 1)
    EGB_BUF(int, status)
    EGB_BUF(double, tune)   // eigenpair scratch of the autotuner's trial solves
#undef EGB_BUF
    double *outs_host = nullptr;  // pinned
    size_t outs_host_cap = 0;
    int *status_host = nullptr;   // pinned
};

#define BCK(...)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (__VA_ARGS__);                                                    \
        if (_e != cudaSuccess)                                                             \
            return set_error(h, ELSI_ERR_CUDA, "%s failed: %s", #__VA_ARGS__,              \
                             cudaGetErrorString(_e));                                      \
    } while (0)

#define BENSURE(name, type, count)                                                         \
    if (!ensure_buf((void **)&b.name, &b.name##_cap, sizeof(type) * (size_t)(count)))     \
        return set_error(h, ELSI_ERR_NOMEM, "cannot allocate batch %s (%zu bytes)", #name,  \
                         sizeof(type) * (size_t)(count));

// ---- autotuner table: per device, precision route, real/complex and size bucket
struct TuneVal {
    int band = 64, solver = 2, workers = 1;
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, TuneVal> g_tune;

static int size_bucket(size_t N)
{
    int q = 0;
    while (((size_t)1 << q) < N) ++q;
    return q;
}

static bool tune_get(int dev, int prec, bool cplx, int bucket, TuneVal *v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, prec, cplx ? 1 : 0, bucket));
    if (it == g_tune.end()) return false;
    *v = it->second;
    return true;
}

static void tune_put(int dev, int prec, bool cplx, int bucket, const TuneVal &v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple(dev, prec, cplx ? 1 : 0, bucket)] = v;
}

bool batch_tuning_lookup(elsi_gb_handle_s *h, int n, bool cplx, int *band, int *solver, int *workers)
{
    int dev = 0;
    cudaGetDevice(&dev);
    TuneVal v;
    if (!tune_get(dev, h->precision, cplx, size_bucket((size_t)(cplx ? 2 : 1) * n), &v)) return false;
    *band = v.band;
    *solver = v.solver;
    *workers = v.workers;
    return true;
}

// Concurrency without tuning: 4 instances for real-form sizes up to 4096, 2 up to 8192.
static int default_workers(size_t N) { return N <= 4096 ? 4 : (N <= 8192 ? 2 : 1); }

// Device memory of one solver instance for real-form size N (workspace of ensure_workspace
// plus the real-form copies of a complex problem), an upper estimate.
static double instance_bytes(size_t N, int prec)
{
    const double n2 = (double)N * (double)N;
    return (prec == ELSI_PREC_FP32_REFINE ? 150.0 : 80.0) * n2 + 64.0 * 1048576.0;
}

static BatchState *batch_state(elsi_gb_handle_s *h)
{
    if (!h->batch) {
        h->batch = new (std::nothrow) BatchState();
        if (!h->batch) return nullptr;
    }
    BatchState &b = *h->batch;
    if (!b.sub) {
        b.sub = new (std::nothrow) elsi_gb_handle_s();
        if (!b.sub) return nullptr;
        b.sub->magic = kHandleMagic;
    }
    return h->batch;
}

static int ensure_small(elsi_gb_handle_s *h, BatchState &b, int nprob)
{
    BENSURE(outs, double, 2 * (size_t)nprob + 8);
    BENSURE(offs, int, (size_t)nprob + 1);
    BENSURE(status, int, ST_WORDS);
    if (b.outs_host_cap < b.outs_cap) {
        if (b.outs_host) cudaFreeHost(b.outs_host);
        b.outs_host = nullptr;
        b.outs_host_cap = 0;
        if (cudaMallocHost((void **)&b.outs_host, b.outs_cap) != cudaSuccess)
            return set_error(h, ELSI_ERR_NOMEM, "pinned batch scalars");
        b.outs_host_cap = b.outs_cap;
    }
    if (!b.status_host && cudaMallocHost((void **)&b.status_host, sizeof(int) * ST_WORDS) != cudaSuccess)
        return set_error(h, ELSI_ERR_NOMEM, "pinned batch status");
    return ELSI_OK;
}

// Reads the batch status word after a stream sync; maps a device error to a return code.
static int batch_status(elsi_gb_handle_s *h, BatchState &b, const char *what)
{
    cudaStream_t st = h->stream;
    BCK(cudaMemcpyAsync(b.status_host, b.status, sizeof(int) * ST_WORDS, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    const int code = b.status_host[ST_CODE];
    if (code == ELSI_ERR_ARG) return set_error(h, code, "%s: electron count outside [0, 2 sum(weights)]", what);
    if (code) return set_error(h, code, "%s: device error %d (aux %d)", what, code, b.status_host[ST_AUX]);
    return ELSI_OK;
}

int batch_ev(elsi_gb_handle_s *h, int nprob, const int *n_basis, const int *n_state,
             const double *const *ham, const double *const *ovlp, bool cplx, double *eval)
{
    if (nprob < 1 || !n_basis || !n_state || !ham)
        return set_error(h, ELSI_ERR_ARG, "batch: nprob < 1 or null array");
    for (int i = 0; i < nprob; ++i) {
        if (n_basis[i] < 1 || n_state[i] < 1 || n_state[i] > n_basis[i])
            return set_error(h, ELSI_ERR_ARG, "batch: problem %d has n_basis %d, n_state %d", i,
                             n_basis[i], n_state[i]);
        if (!ham[i]) return set_error(h, ELSI_ERR_ARG, "batch: problem %d has no Hamiltonian", i);
        if (!h->overlap_is_unit && (!ovlp || !ovlp[i]))
            return set_error(h, ELSI_ERR_ARG, "batch: problem %d has no overlap", i);
    }
    BatchState *bp = batch_state(h);
    if (!bp) return set_error(h, ELSI_ERR_NOMEM, "batch state");
    BatchState &b = *bp;
    b.items.assign(nprob, BatchItem());
    b.cplx = cplx;
    size_t nval = 0, nvec = 0, nlvl = 0, max_nk = 0, max_nn = 0;
    for (int i = 0; i < nprob; ++i) {
        BatchItem &it = b.items[i];
        it.n = n_basis[i];
        it.k = n_state[i];
        const size_t N = cplx ? 2 * (size_t)it.n : it.n, K = cplx ? 2 * (size_t)it.k : it.k;
        it.off_val = nval;
        it.off_vec = nvec;
        it.off_lvl = nlvl;
        nval += N;
        nvec += N * K;
        nlvl += it.k;
        if (N * K > max_nk) max_nk = N * K;
        if (N * N > max_nn) max_nn = N * N;
    }
    b.total_lvl = nlvl;
    BENSURE(vals, double, nval);
    BENSURE(vecs, double, nvec);
    BENSURE(lvl, double, nlvl);
    BENSURE(wts, double, nlvl);
    BENSURE(occ, double, nlvl);
    BENSURE(cw, double, max_nk);
    if (cplx) {
        BENSURE(emb, double, 2 * max_nn);
        size_t kmax = 0;
        for (auto &it : b.items) kmax = it.k > (int)kmax ? it.k : kmax;
        BENSURE(occ2, double, 2 * kmax);
    }
    int rc = ensure_small(h, b, nprob);
    if (rc) return rc;
    {
        std::vector<int> off(nprob + 1);
        for (int i = 0; i < nprob; ++i) off[i] = (int)b.items[i].off_lvl;
        off[nprob] = (int)nlvl;
        BCK(cudaMemcpyAsync(b.offs, off.data(), sizeof(int) * (nprob + 1), cudaMemcpyHostToDevice, h->stream));
        BCK(cudaStreamSynchronize(h->stream));
    }
    // Problem order: largest first (longest-processing-time order), each problem taken by
    // the next free solver instance (worker: own handle, stream and host thread, since a
    // solve is synchronous on its host thread).
    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = i;
    const int mult = cplx ? 2 : 1;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b.items[x].n > b.items[y].n; });
    cudaStream_t st = h->stream;
    BCK(cudaStreamSynchronize(st));  // inputs produced on the caller's stream are ready
    int dev = 0;
    cudaGetDevice(&dev);

    // the configuration of one solve: route settings of the handle, reduction of the tuner
    auto configure = [&](elsi_gb_handle_s *s, cudaStream_t wst, const TuneVal &tv) {
        s->overlap_is_unit = h->overlap_is_unit;
        s->scheme = h->scheme;
        s->kt = h->kt;
        s->occ_accuracy = h->occ_accuracy;
        s->mu_max_steps = h->mu_max_steps;
        s->precision = h->precision;
        s->band_width = tv.band;
        s->elpa_solver = tv.solver;
        s->refine_max_iter = h->refine_max_iter;
        s->stream = wst;
        s->reuse_l = false;
        s->occ_stride = cplx ? 2 : 1;
    };
    struct Result {
        int rc = ELSI_OK;
        std::string msg;
        float stage_ms[kNumStages] = {};
        int refine_min = 1 << 30;
        double orth_max = 0.0;
    };
    // solve problem i in instance s on stream wst; eigenpairs to (vals, vecs)
    auto solve_one = [&](elsi_gb_handle_s *s, cudaStream_t wst, int i, const TuneVal &tv,
                         double *vals, double *vecs, Result &r) -> bool {
        const BatchItem &it = b.items[i];
        const size_t N = (size_t)mult * it.n;
        configure(s, wst, tv);
        s->n = (int)N;
        s->n_state = mult * it.k;
        s->n_electron = 0.0;
        s->have_l = false;
        SolveRequest rq;
        rq.ham = ham[i];
        rq.ovlp = h->overlap_is_unit ? nullptr : ovlp[i];
        cudaError_t ce = cudaSuccess;
        if (cplx) {
            Workspace &sw = s->wk;
            if (!ensure_buf((void **)&sw.host_h, &sw.host_h_cap, sizeof(double) * N * N) ||
                (rq.ovlp && !ensure_buf((void **)&sw.host_s, &sw.host_s_cap, sizeof(double) * N * N))) {
                r.rc = ELSI_ERR_NOMEM;
                r.msg = "batch: real-form buffers";
                return false;
            }
            ce = embed_hermitian(wst, it.n, ham[i], sw.host_h);
            if (ce == cudaSuccess && rq.ovlp) ce = embed_hermitian(wst, it.n, ovlp[i], sw.host_s);
            rq.ham = sw.host_h;
            rq.ovlp = rq.ovlp ? sw.host_s : nullptr;
        }
        if (ce != cudaSuccess) {
            r.rc = ELSI_ERR_CUDA;
            r.msg = cudaGetErrorString(ce);
            return false;
        }
        rq.eval = vals;
        rq.evec = vecs;
        const int rc2 = run_solve(s, rq);
        if (rc2) {
            r.rc = rc2;
            r.msg = "batch problem " + std::to_string(i) + ": " + s->last_error;
            return false;
        }
        return true;
    };
    auto instance = [&](int t, elsi_gb_handle_s **s, cudaStream_t *wst) {
        *s = (t == 0) ? b.sub : b.workers[t - 1].sub;
        *wst = (t == 0) ? st : b.workers[t - 1].stream;
    };
    auto add_workers = [&](int W) -> int {
        while ((int)b.workers.size() < W - 1) {
            BatchWorker wk;
            wk.sub = new (std::nothrow) elsi_gb_handle_s();
            if (!wk.sub) return set_error(h, ELSI_ERR_NOMEM, "batch worker");
            wk.sub->magic = kHandleMagic;
            if (cudaStreamCreateWithFlags(&wk.stream, cudaStreamNonBlocking) != cudaSuccess) {
                delete wk.sub;
                return set_error(h, ELSI_ERR_CUDA, "batch worker stream");
            }
            b.workers.push_back(wk);
        }
        return ELSI_OK;
    };
    // upper bound of concurrent instances for real-form size N from the free device memory
    auto mem_workers = [&](size_t N) -> int {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 1;
        const double per = instance_bytes(N, h->precision);
        int wm = (int)(0.8 * (double)fr / per) + (int)b.workers.size() + 1;
        return wm < 1 ? 1 : (wm > 16 ? 16 : wm);
    };

    // ---- tuning of one size bucket on its first problem i (real-form size N): the
    // reduction variant with the shortest solve, then the concurrency with the highest
    // throughput (each instance solves problem i into its own scratch; the times of the
    // second of two runs count, so that workspace allocation is excluded)
    auto tune_bucket = [&](int i, size_t N, TuneVal &best) -> int {
        const BatchItem &it = b.items[i];
        const size_t K = (size_t)mult * it.k;
        const int wmax = h->batch_workers > 0 ? h->batch_workers : mem_workers(N);
        BENSURE(tune, double, (size_t)(wmax > 16 ? 16 : wmax) * (N + N * K));
        auto scratch = [&](int t, double **vals, double **vecs) {
            *vals = b.tune + (size_t)t * (N + N * K);
            *vecs = *vals + N;
        };
        auto run_concurrent = [&](int W, const TuneVal &v, double *secs) -> int {
            int rc = add_workers(W);
            if (rc) return rc;
            std::vector<Result> rr(W);
            for (int rep = 0; rep < 2; ++rep) {
                const auto t0 = std::chrono::steady_clock::now();
                std::vector<std::thread> th;
                auto one = [&](int t) {
                    cudaSetDevice(dev);
                    elsi_gb_handle_s *s;
                    cudaStream_t wst;
                    instance(t, &s, &wst);
                    double *vals, *vecs;
                    scratch(t, &vals, &vecs);
                    if (solve_one(s, wst, i, v, vals, vecs, rr[t])) {
                        const cudaError_t ce = cudaStreamSynchronize(wst);
                        if (ce != cudaSuccess && rr[t].rc == ELSI_OK) {
                            rr[t].rc = ELSI_ERR_CUDA;
                            rr[t].msg = cudaGetErrorString(ce);
                        }
                    }
                };
                for (int t = 1; t < W; ++t) th.emplace_back(one, t);
                one(0);
                for (auto &x : th) x.join();
                *secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                for (int t = 0; t < W; ++t)
                    if (rr[t].rc) return set_error(h, rr[t].rc, "%s", rr[t].msg.c_str());
            }
            return ELSI_OK;
        };
        // reduction variants (those set explicitly on the handle are kept)
        std::vector<TuneVal> cand;
        const int bands[2] = {32, 64};
        for (int bw : bands)
            if (!h->band_set || bw == h->band_width)
                if (!h->solver_set || h->elpa_solver == 2) cand.push_back(TuneVal{bw, 2, 1});
        if (!h->solver_set || h->elpa_solver == 1) cand.push_back(TuneVal{h->band_width, 1, 1});
        if (cand.empty()) cand.push_back(TuneVal{h->band_width, h->elpa_solver, 1});
        double tbest = 1e300;
        for (const TuneVal &c : cand) {
            double sec = 0.0;
            int rc = run_concurrent(1, c, &sec);
            if (rc) return rc;
            if (sec < tbest) { tbest = sec; best.band = c.band; best.solver = c.solver; }
        }
        // concurrency
        best.workers = 1;
        if (h->batch_workers > 0) {
            best.workers = h->batch_workers;
        } else {
            double thr_best = 1.0 / tbest;
            for (int W = 2; W <= wmax && W <= 16; W *= 2) {
                double sec = 0.0;
                int rc = run_concurrent(W, best, &sec);
                if (rc) return rc;
                const double thr = W / sec;
                if (thr > 1.05 * thr_best) { thr_best = thr; best.workers = W; }
                else break;
            }
        }
        return ELSI_OK;
    };

    // ---- autotuning of the size buckets met for the first time
    const int prec = h->precision;
    std::vector<TuneVal> tv(nprob);
    for (int q = 0; q < nprob; ++q) {
        const int i = order[q];
        const size_t N = (size_t)mult * b.items[i].n;
        TuneVal v;
        const bool known = tune_get(dev, prec, cplx, size_bucket(N), &v);
        if (!known) {
            v.band = h->band_width;
            v.solver = h->elpa_solver;
            v.workers = h->batch_workers > 0 ? h->batch_workers : default_workers(N);
            if (h->batch_autotune) {
                int rc = tune_bucket(i, N, v);
                if (rc) return rc;
            }
            tune_put(dev, prec, cplx, size_bucket(N), v);
        }
        if (h->band_set) v.band = h->band_width;
        if (h->solver_set) v.solver = h->elpa_solver;
        tv[i] = v;
    }

    // ---- the batch: concurrency of the bucket with the most work, bounded by memory
    int W = 1;
    {
        double wbest = -1.0;
        size_t nmax = 0;
        std::map<int, double> work;
        for (int i = 0; i < nprob; ++i) {
            const double N = (double)mult * b.items[i].n;
            work[size_bucket((size_t)N)] += N * N * N;
            if ((size_t)N > nmax) nmax = (size_t)N;
        }
        for (int i = 0; i < nprob; ++i) {
            const size_t N = (size_t)mult * b.items[i].n;
            const double wk = work[size_bucket(N)];
            if (wk > wbest) { wbest = wk; W = tv[i].workers; }
        }
        if (h->batch_workers > 0) W = h->batch_workers;
        const int wm = mem_workers(nmax);
        if (W > wm) W = wm;
        if (W > nprob) W = nprob;
        if (W < 1) W = 1;
    }
    rc = add_workers(W);
    if (rc) return rc;
    std::vector<Result> res(W);
    std::atomic<int> next{0};
    auto work = [&](int t) {
        cudaSetDevice(dev);
        elsi_gb_handle_s *s;
        cudaStream_t wst;
        instance(t, &s, &wst);
        Result &r = res[t];
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= nprob) break;
            const int i = order[q];
            const BatchItem &it = b.items[i];
            if (!solve_one(s, wst, i, tv[i], b.vals + it.off_val, b.vecs + it.off_vec, r)) {
                next.store(nprob);  // the other instances stop after their current problem
                return;
            }
            const cudaError_t ce = cplx ? pair_evals(wst, it.k, b.vals + it.off_val, b.lvl + it.off_lvl)
                                        : cudaMemcpyAsync(b.lvl + it.off_lvl, b.vals + it.off_val,
                                                          sizeof(double) * it.k, cudaMemcpyDeviceToDevice, wst);
            if (ce != cudaSuccess) {
                r.rc = ELSI_ERR_CUDA;
                r.msg = cudaGetErrorString(ce);
                next.store(nprob);
                return;
            }
            for (int q2 = 0; q2 < kNumStages; ++q2) r.stage_ms[q2] += s->stage_ms[q2];
            if (s->refine_iters < r.refine_min) r.refine_min = s->refine_iters;
            if (s->orth_err > r.orth_max) r.orth_max = s->orth_err;
        }
        const cudaError_t ce = cudaStreamSynchronize(wst);
        if (ce != cudaSuccess && r.rc == ELSI_OK) {
            r.rc = ELSI_ERR_CUDA;
            r.msg = cudaGetErrorString(ce);
        }
    };
    {
        std::vector<std::thread> threads;
        for (int t = 1; t < W; ++t) threads.emplace_back(work, t);
        work(0);
        for (auto &th : threads) th.join();
    }
    float stage_ms[kNumStages] = {};
    int refine_min = 1 << 30;
    double orth_max = 0.0;
    for (int t = 0; t < W; ++t) {
        if (res[t].rc) return set_error(h, res[t].rc, "%s", res[t].msg.c_str());
        for (int q = 0; q < kNumStages; ++q) stage_ms[q] += res[t].stage_ms[q];
        refine_min = res[t].refine_min < refine_min ? res[t].refine_min : refine_min;
        orth_max = res[t].orth_max > orth_max ? res[t].orth_max : orth_max;
    }
    if (eval) BCK(cudaMemcpyAsync(eval, b.lvl, sizeof(double) * nlvl, cudaMemcpyDeviceToDevice, st));
    BCK(cudaStreamSynchronize(st));
    for (int q = 0; q < kNumStages; ++q) h->stage_ms[q] = stage_ms[q];
    h->refine_iters = refine_min;
    h->orth_err = orth_max;
    h->have_edm = h->have_occ = h->have_cedm = false;
    return ELSI_OK;
}

int batch_occupation(elsi_gb_handle_s *h, int m, const double *eps, const double *wt, double n_el,
                     double *occ, double *mu)
{
    BatchState *bp = batch_state(h);
    if (!bp) return set_error(h, ELSI_ERR_NOMEM, "batch state");
    BatchState &b = *bp;
    int rc = ensure_small(h, b, b.items.empty() ? 1 : (int)b.items.size());
    if (rc) return rc;
    cudaStream_t st = h->stream;
    BCK(cudaMemsetAsync(b.status, 0, sizeof(int) * ST_WORDS, st));
    BCK(occupation_weighted(st, m, eps, wt, n_el, h->scheme, h->kt, h->occ_accuracy,
                            h->mu_max_steps, occ, b.outs, b.status));
    BCK(cudaMemcpyAsync(b.outs_host, b.outs, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
    rc = batch_status(h, b, "weighted occupation");
    if (rc) return rc;
    if (mu) *mu = b.outs_host[0];
    h->mu = b.outs_host[0];
    return ELSI_OK;
}

int batch_dm(elsi_gb_handle_s *h, const double *occ, double *const *dm, double *const *edm,
             double *energy)
{
    BatchState *bp = h->batch;
    if (!bp || bp->items.empty()) return set_error(h, ELSI_ERR_STATE, "no batched eigensolve yet");
    if (!dm) return set_error(h, ELSI_ERR_ARG, "batch: null density-matrix array");
    BatchState &b = *bp;
    const int nprob = (int)b.items.size();
    for (int i = 0; i < nprob; ++i)
        if (!dm[i]) return set_error(h, ELSI_ERR_ARG, "batch: problem %d has no density-matrix buffer", i);
    cudaStream_t st = h->stream;
    if (occ && occ != b.occ)
        BCK(cudaMemcpyAsync(b.occ, occ, sizeof(double) * b.total_lvl, cudaMemcpyDeviceToDevice, st));
    for (int i = 0; i < nprob; ++i) {
        const BatchItem &it = b.items[i];
        double *w_out = (edm && edm[i]) ? edm[i] : nullptr;
        if (!b.cplx) {
            BCK(density_pw<double>(st, it.n, it.k, b.vecs + it.off_vec, it.n, b.occ + it.off_lvl,
                                   b.vals + it.off_val, dm[i], w_out, b.cw));
        } else {
            const int N = 2 * it.n, K = 2 * it.k;
            double *pe = b.emb, *we = b.emb + (size_t)N * N;
            BCK(dup_pairs(st, it.k, b.occ + it.off_lvl, b.occ2));
            BCK(density_pw<double>(st, N, K, b.vecs + it.off_vec, N, b.occ2, b.vals + it.off_val,
                                   pe, w_out ? we : nullptr, b.cw));
            BCK(fold_hermitian(st, it.n, pe, dm[i]));
            if (w_out) BCK(fold_hermitian(st, it.n, we, w_out));
        }
    }
    BCK(segment_energy(st, nprob, b.offs, b.occ, b.lvl, b.outs));
    BCK(cudaMemcpyAsync(b.outs_host, b.outs, sizeof(double) * nprob, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    if (energy)
        for (int i = 0; i < nprob; ++i) energy[i] = b.outs_host[i];
    return ELSI_OK;
}

int dm_batched(elsi_gb_handle_s *h, int nprob, const int *n_basis, const int *n_state,
               const double *const *ham, const double *const *ovlp, const double *weight,
               const double *n_electron, int shared_mu, double *const *dm, double *const *edm,
               double *energy, double *mu, bool cplx)
{
    if (!n_electron || !dm) return set_error(h, ELSI_ERR_ARG, "batch: null array");
    if (shared_mu && !weight) return set_error(h, ELSI_ERR_ARG, "batch: shared mu needs weights");
    int rc = batch_ev(h, nprob, n_basis, n_state, ham, ovlp, cplx, nullptr);
    if (rc) return rc;
    BatchState &b = *h->batch;
    cudaStream_t st = h->stream;
    if (shared_mu) {
        std::vector<double> w(b.total_lvl);
        for (int i = 0; i < nprob; ++i) {
            if (!(weight[i] >= 0.0)) return set_error(h, ELSI_ERR_ARG, "batch: weight %d negative", i);
            for (int l = 0; l < b.items[i].k; ++l) w[b.items[i].off_lvl + l] = weight[i];
        }
        BCK(cudaMemcpyAsync(b.wts, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, st));
        double m = 0.0;
        rc = batch_occupation(h, (int)b.total_lvl, b.lvl, b.wts, n_electron[0], b.occ, &m);
        if (rc) return rc;
        if (mu) mu[0] = m;
    } else {
        for (int i = 0; i < nprob; ++i)
            if (!(n_electron[i] >= 0.0) || n_electron[i] > 2.0 * b.items[i].k)
                return set_error(h, ELSI_ERR_ARG, "batch: problem %d has %g electrons for %d states",
                                 i, n_electron[i], b.items[i].k);
        BCK(cudaMemsetAsync(b.status, 0, sizeof(int) * ST_WORDS, st));
        for (int i = 0; i < nprob; ++i) {
            const BatchItem &it = b.items[i];
            BCK(occupation(st, it.k, b.lvl + it.off_lvl, n_electron[i], h->scheme, h->kt,
                           h->occ_accuracy, h->mu_max_steps, b.occ + it.off_lvl, b.outs + 2 * i,
                           b.status, 1));
        }
        BCK(cudaMemcpyAsync(b.outs_host, b.outs, sizeof(double) * 2 * nprob, cudaMemcpyDeviceToHost, st));
        rc = batch_status(h, b, "occupation");
        if (rc) return rc;
        if (mu)
            for (int i = 0; i < nprob; ++i) mu[i] = b.outs_host[2 * i];
    }
    return batch_dm(h, nullptr, dm, edm, energy);
}

void free_batch(elsi_gb_handle_s *h)
{
    if (!h->batch) return;
    BatchState &b = *h->batch;
    void *bufs[] = {b.vals, b.vecs, b.lvl, b.wts, b.occ, b.occ2, b.emb, b.cw, b.outs, b.offs, b.status,
                    b.tune};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b.outs_host) cudaFreeHost(b.outs_host);
    if (b.status_host) cudaFreeHost(b.status_host);
    if (b.sub) {
        free_complex(b.sub);
        free_workspace(b.sub);
        delete b.sub;
    }
    for (auto &wk : b.workers) {
        if (wk.sub) {
            free_complex(wk.sub);
            free_workspace(wk.sub);
            delete wk.sub;
        }
        if (wk.stream) cudaStreamDestroy(wk.stream);
    }
    delete h->batch;
    h->batch = nullptr;
}

int batch_levels(elsi_gb_handle_s *h) { return h->batch ? (int)h->batch->total_lvl : 0; }

}  // namespace egb
