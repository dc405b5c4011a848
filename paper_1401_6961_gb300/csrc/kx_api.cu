// kx_api.cu -- the C ABI declared in include/kx.h.  Argument checks, call
// order, device selection and host marshalling live here; every step of the
// computation runs in the kernels of the other translation units.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "kx_internal.cuh"

using namespace kx;

namespace {

// Makes the context's device current for the duration of a call and puts
// the caller's device back afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
        if (!ok) (void)cudaGetLastError();
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

__global__ void k_filter_work(const Task* __restrict__ w, int64_t n, const uint8_t* __restrict__ amark,
                              Task* __restrict__ out, unsigned long long* __restrict__ cnt, int64_t cap) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Task t = w[i];
        if (amark && !amark[t.a]) continue;
        unsigned long long pos = atomicAdd(cnt, 1ull);
        if ((int64_t)pos < cap) out[pos] = t;
    }
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// tree position of the shell of every function (user order), for the
// mirror of a symmetric build
int function_positions(kx_ctx* c) {
    std::vector<int32_t> inv(c->n_shell), f((size_t)c->n_fn);
    for (int i = 0; i < c->n_shell; ++i) inv[c->perm[i]] = i;
    for (int s = 0; s < c->n_shell; ++s)
        for (int64_t m = c->fn_off[s]; m < c->fn_off[s + 1]; ++m) f[m] = inv[s];
    if (!c->d_ftpos) KX_CUDA(c, cudaMalloc(&c->d_ftpos, sizeof(int32_t) * c->n_fn));
    KX_CUDA(c, cudaMemcpy(c->d_ftpos, f.data(), sizeof(int32_t) * c->n_fn, cudaMemcpyHostToDevice));
    return KX_OK;
}

int check_ctx(const kx_ctx* c) { return c ? KX_OK : KX_EINVAL; }

void free_all(kx_ctx* c) {
    drop_graph(c);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->h_gw) cudaFreeHost(c->h_gw);
    c->gstream = nullptr;
    c->h_gw = nullptr;
    void* ptrs[] = {c->d_tl, c->d_tctr, c->d_talpha, c->d_tfoff, c->d_perm, c->d_s2, c->d_snorm, c->d_slog,
                    c->d_pq, c->d_pnorm, c->d_plog, c->d_node_lo, c->d_node_hi, c->d_node_child,
                    c->d_node_nchild, c->d_sq_s, c->d_sq_p, c->d_nrm_s, c->d_nrm_p, c->d_leaf_lo, c->d_leaf_hi,
                    c->d_boys64, c->d_boys32, c->d_pairmap, c->d_scratch, c->d_front[0], c->d_front[1],
                    c->d_mask, c->d_scan, c->d_rec, c->d_bin, c->d_counters, c->d_keep, c->d_P32, c->d_scantmp,
                    c->d_hostP, c->d_hostK, c->d_leafdesc, c->d_list, c->d_sseg, c->d_tsys, c->d_lseg,
                    c->d_node_sys, c->d_mframe, c->d_gw, c->d_groots, c->d_gactive, c->d_tuneK,
                    c->d_fseg, c->d_ftpos, c->d_boysdw, c->d_Pdw, c->d_work, c->d_sflops};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < NPAIRCLASS; ++i) {
        if (c->d_pairmeta[i]) cudaFree(c->d_pairmeta[i]);
        if (c->d_pair64[i]) cudaFree(c->d_pair64[i]);
        if (c->d_pair32[i]) cudaFree(c->d_pair32[i]);
        if (c->d_pairdw[i]) cudaFree(c->d_pairdw[i]);
    }
}

}  // namespace

extern "C" {

void kx_default_opts(kx_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tau = 1e-10;
    o->split_threshold = 1e-5;
    o->precision = KX_FP64;
    o->shell_screen = 1;
    o->keep_worklist = 0;
    o->profile = 0;
    o->chunk_records = 0;
    o->symmetric = 0;
    o->reserved = 0;
}

int kx_create_batch(kx_ctx** out, int32_t n_sys, const kx_basis* bases, int device, void* cuda_stream) {
    if (!out) return KX_EINVAL;
    *out = nullptr;
    if (!bases || n_sys < 1 || n_sys > 65535) return KX_EINVAL;
    int64_t tot_atom = 0, tot_shell = 0, tot_fn = 0;
    for (int y = 0; y < n_sys; ++y) {
        const kx_basis* b = bases + y;
        if (!b->xyz || !b->shell_atom || !b->shell_l || !b->shell_alpha) return KX_EINVAL;
        if (b->n_atom <= 0 || b->n_shell <= 0 || b->n_shell > 65535) return KX_EINVAL;
        for (int i = 0; i < 3 * b->n_atom; ++i)
            if (!std::isfinite(b->xyz[i])) return KX_EINVAL;
        for (int s = 0; s < b->n_shell; ++s) {
            if (b->shell_atom[s] < 0 || b->shell_atom[s] >= b->n_atom) return KX_EINVAL;
            if (b->shell_l[s] < 0 || b->shell_l[s] > LMAX) return KX_EINVAL;
            if (!finite_pos(b->shell_alpha[s])) return KX_EINVAL;
            tot_fn += ncart(b->shell_l[s]);
        }
        tot_atom += b->n_atom;
        tot_shell += b->n_shell;
    }
    if (tot_shell > (1 << 24) || tot_atom > (1 << 24) || tot_fn > ((int64_t)1 << 30)) return KX_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        (void)cudaGetLastError();
        return KX_ECUDA;
    }
    kx_ctx* c = new (std::nothrow) kx_ctx();
    if (!c) return KX_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    if (!g.ok) {
        delete c;
        return KX_ECUDA;
    }
    // concatenate the systems: atoms, shells and functions system-major
    c->n_sys = n_sys;
    c->n_atom = (int)tot_atom;
    c->n_shell = (int)tot_shell;
    c->sys_atom.assign(n_sys + 1, 0);
    c->sys_shell.assign(n_sys + 1, 0);
    c->sys_fn.assign(n_sys + 1, 0);
    c->sys_mat.assign(n_sys + 1, 0);
    c->sseg.resize(n_sys);
    c->fn_off.assign(1, 0);
    for (int y = 0; y < n_sys; ++y) {
        const kx_basis* b = bases + y;
        const int a0 = c->sys_atom[y];
        c->xyz.insert(c->xyz.end(), b->xyz, b->xyz + 3 * (size_t)b->n_atom);
        for (int s = 0; s < b->n_shell; ++s) {
            c->shell_atom.push_back(a0 + b->shell_atom[s]);
            c->shell_l.push_back(b->shell_l[s]);
            c->shell_alpha.push_back(b->shell_alpha[s]);
            c->fn_off.push_back(c->fn_off.back() + ncart(b->shell_l[s]));
        }
        c->sys_atom[y + 1] = a0 + b->n_atom;
        c->sys_shell[y + 1] = c->sys_shell[y] + b->n_shell;
        c->sys_fn[y + 1] = c->fn_off.back();
        const int64_t nf = c->sys_fn[y + 1] - c->sys_fn[y];
        c->sys_mat[y + 1] = c->sys_mat[y] + nf * nf;
        c->sseg[y] = Seg{c->sp_total, c->sys_shell[y], b->n_shell};
        c->sp_total += (int64_t)b->n_shell * b->n_shell;
    }
    c->n_fn = c->fn_off.back();
    for (int s = 0; s < NSTREAM; ++s) {
        c->eri_threads[s] = ERI_THREADS;
        c->eri_bpsm[s] = 0;
        c->eri_variant[s] = 0;
    }
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->n_sm < 1) {
        (void)cudaGetLastError();
        c->n_sm = 0;
    }
    std::vector<int32_t> tsys(c->n_shell);
    for (int y = 0; y < n_sys; ++y)
        for (int i = c->sys_shell[y]; i < c->sys_shell[y + 1]; ++i) tsys[i] = y;
    int r = KX_OK;
    cudaError_t e = cudaMalloc(&c->d_counters, sizeof(unsigned long long) * NCOUNTERS);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * NCOUNTERS, c->stream);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_sseg, sizeof(Seg) * n_sys);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tsys, sizeof(int32_t) * c->n_shell);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_sseg, c->sseg.data(), sizeof(Seg) * n_sys, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_tsys, tsys.data(), sizeof(int32_t) * c->n_shell, cudaMemcpyHostToDevice, c->stream);
    std::vector<Seg> fseg(n_sys);
    for (int y = 0; y < n_sys; ++y)
        fseg[y] = Seg{c->sys_mat[y], (int32_t)c->sys_fn[y], (int32_t)(c->sys_fn[y + 1] - c->sys_fn[y])};
    if (e == cudaSuccess) e = cudaMalloc(&c->d_fseg, sizeof(Seg) * n_sys);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_fseg, fseg.data(), sizeof(Seg) * n_sys, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) r = cuda_check(c, e, "kx_create");
    if (r == KX_OK && c->n_sm < 1) r = set_err(c, KX_ECUDA, "multiprocessor count query failed");
    if (r == KX_OK) r = boys_table(c);
    if (r == KX_OK) r = order_atoms(c);
    if (r == KX_OK) r = function_positions(c);
    if (r != KX_OK) {
        free_all(c);
        delete c;
        return r;
    }
    *out = c;
    return KX_OK;
}

int kx_create(kx_ctx** out, const kx_basis* b, int device, void* cuda_stream) {
    return kx_create_batch(out, 1, b, device, cuda_stream);
}

int kx_build_schwarz(kx_ctx* c, double tau_ovlp) {
    KX_TRY(check_ctx(c));
    if (!std::isfinite(tau_ovlp) || tau_ovlp < 0.0) return set_err(c, KX_EINVAL, "tau_ovlp must be >= 0");
    if (!c->have_order) return set_err(c, KX_ESTATE, "no shell order");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    c->tau_ovlp = tau_ovlp;
    c->have_tree = false;
    drop_graph(c);
    return schwarz(c, tau_ovlp);
}

int kx_build_tree(kx_ctx* c, int32_t leaf_max_functions, const int32_t* perm) {
    KX_TRY(check_ctx(c));
    if (leaf_max_functions < 1) return set_err(c, KX_EINVAL, "leaf_max_functions must be >= 1");
    if (!c->have_schwarz) return set_err(c, KX_ESTATE, "kx_build_schwarz must come first");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    if (perm) {
        std::vector<char> seen(c->n_shell, 0);
        for (int i = 0; i < c->n_shell; ++i) {
            if (perm[i] < 0 || perm[i] >= c->n_shell || seen[perm[i]])
                return set_err(c, KX_EINVAL, "perm is not a permutation of the shells");
            seen[perm[i]] = 1;
        }
        // a batch keeps every system's shells in its own range of tree positions
        for (int y = 0; y < c->n_sys; ++y) {
            for (int i = c->sys_shell[y]; i < c->sys_shell[y + 1]; ++i)
                if (perm[i] < c->sys_shell[y] || perm[i] >= c->sys_shell[y + 1])
                    return set_err(c, KX_EINVAL, "perm moves a shell out of its system");
        }
        c->perm.assign(perm, perm + c->n_shell);
        KX_CUDA(c, cudaMemcpyAsync(c->d_perm, c->perm.data(), sizeof(int32_t) * c->n_shell,
                                   cudaMemcpyHostToDevice, c->stream));
        // the Schwarz table is kept in tree order: rebuild it for the new order
        KX_TRY(schwarz(c, c->tau_ovlp));
        KX_TRY(function_positions(c));
    }
    c->have_tree = false;
    c->keep_valid = false;
    drop_graph(c);
    return build_tree(c, leaf_max_functions);
}

}  // extern "C"

namespace {

// ldp = ldk = 0: P and K packed per system (the batch entry points)
int exchange_impl(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
                  kx_stats* st) {
    if (!P || !K || !o) return set_err(c, KX_EINVAL, "null argument");
    if (!std::isfinite(o->tau) || o->tau < 0.0) return set_err(c, KX_EINVAL, "tau must be >= 0");
    if (o->precision < KX_FP64 || o->precision > KX_MIXED_DW) return set_err(c, KX_EINVAL, "bad precision");
    if (o->precision != KX_FP64 && (!std::isfinite(o->split_threshold) || o->split_threshold < 0.0))
        return set_err(c, KX_EINVAL, "split_threshold must be >= 0");
    if (o->chunk_records < 0) return set_err(c, KX_EINVAL, "chunk_records must be >= 0");
    if (o->symmetric != 0 && o->symmetric != 1) return set_err(c, KX_EINVAL, "symmetric must be 0 or 1");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    if (!std::isfinite(o->split_budget) || o->split_budget < 0.0)
        return set_err(c, KX_EINVAL, "split_budget must be >= 0");
    kx_stats local;
    kx_stats* s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    // a split from the error budget: plan first, then build with it
    kx_opts ob = *o;
    kx_stats sp;
    std::memset(&sp, 0, sizeof(sp));
    if (o->precision != KX_FP64 && o->split_budget > 0.0) {
        KX_TRY(split_plan(c, P, ldp, o, o->split_budget, &sp));
        ob.split_threshold = sp.split_used;
        ob.split_budget = 0.0;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    int r = traverse_and_evaluate(c, P, ldp, &ob, K, ldk, s);
    s->split_used = o->precision != KX_FP64 ? ob.split_threshold : 0.0;
    s->fp32_err_estimate = sp.fp32_err_estimate;
    s->fp32_err_bound = sp.fp32_err_bound;
    cudaEventRecord(e1, c->stream);
    if (r == KX_OK) {
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) r = cuda_check(c, e, "kx_exchange");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        s->ms_total = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
}

}  // namespace

extern "C" {

int kx_exchange(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
                kx_stats* st) {
    KX_TRY(check_ctx(c));
    if (!P || !K || !o) return set_err(c, KX_EINVAL, "null argument");
    if (ldp < c->n_fn || ldk < c->n_fn) return set_err(c, KX_EINVAL, "leading dimension smaller than n_fn");
    if (c->n_sys != 1) return set_err(c, KX_EINVAL, "a batch context takes packed P and K (kx_exchange_batch)");
    return exchange_impl(c, P, ldp, o, K, ldk, st);
}

int kx_exchange_host(kx_ctx* c, const double* P_host, int64_t ldp, const kx_opts* o, double* K_host, int64_t ldk,
                     kx_stats* st) {
    KX_TRY(check_ctx(c));
    if (!P_host || !K_host || !o) return set_err(c, KX_EINVAL, "null argument");
    if (ldp < c->n_fn || ldk < c->n_fn) return set_err(c, KX_EINVAL, "leading dimension smaller than n_fn");
    if (c->n_sys != 1) return set_err(c, KX_EINVAL, "a batch context takes packed P and K");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    size_t n = (size_t)c->n_fn;
    if (c->host_cap < n * n) {
        cudaFree(c->d_hostP);
        cudaFree(c->d_hostK);
        c->d_hostP = c->d_hostK = nullptr;
        c->host_cap = 0;
        KX_CUDA(c, cudaMalloc(&c->d_hostP, sizeof(double) * n * n));
        KX_CUDA(c, cudaMalloc(&c->d_hostK, sizeof(double) * n * n));
        c->host_cap = n * n;
    }
    KX_CUDA(c, cudaMemcpy2DAsync(c->d_hostP, sizeof(double) * n, P_host, sizeof(double) * ldp, sizeof(double) * n, n,
                                 cudaMemcpyHostToDevice, c->stream));
    KX_TRY(kx_exchange(c, c->d_hostP, (int64_t)n, o, c->d_hostK, (int64_t)n, st));
    KX_CUDA(c, cudaMemcpy2DAsync(K_host, sizeof(double) * ldk, c->d_hostK, sizeof(double) * n, sizeof(double) * n, n,
                                 cudaMemcpyDeviceToHost, c->stream));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    return KX_OK;
}

int kx_count(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, kx_stats* st) {
    KX_TRY(check_ctx(c));
    if (!P || !o || !st) return set_err(c, KX_EINVAL, "null argument");
    if (c->n_sys == 1 ? ldp < c->n_fn : ldp != 0)
        return set_err(c, KX_EINVAL, "ldp must be >= n_fn (0 for the packed P of a batch)");
    if (!std::isfinite(o->tau) || o->tau < 0.0) return set_err(c, KX_EINVAL, "tau must be >= 0");
    if (o->precision < KX_FP64 || o->precision > KX_MIXED_DW) return set_err(c, KX_EINVAL, "bad precision");
    if (o->precision != KX_FP64 && (!std::isfinite(o->split_threshold) || o->split_threshold < 0.0))
        return set_err(c, KX_EINVAL, "split_threshold must be >= 0");
    if (o->symmetric != 0 && o->symmetric != 1) return set_err(c, KX_EINVAL, "symmetric must be 0 or 1");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    if (!std::isfinite(o->split_budget) || o->split_budget < 0.0)
        return set_err(c, KX_EINVAL, "split_budget must be >= 0");
    std::memset(st, 0, sizeof(*st));
    kx_opts ob = *o;
    kx_stats sp;
    std::memset(&sp, 0, sizeof(sp));
    if (o->precision != KX_FP64 && o->split_budget > 0.0) {
        KX_TRY(split_plan(c, P, ldp, o, o->split_budget, &sp));
        ob.split_threshold = sp.split_used;
        ob.split_budget = 0.0;
    }
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    const int r = drive(c, RUN_COUNT, P, ldp, &ob, nullptr, 0, st, nullptr, 0);
    st->split_used = o->precision != KX_FP64 ? ob.split_threshold : 0.0;
    st->fp32_err_estimate = sp.fp32_err_estimate;
    st->fp32_err_bound = sp.fp32_err_bound;
    return r;
}

int kx_row_work(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double* work) {
    KX_TRY(check_ctx(c));
    if (!work) return set_err(c, KX_EINVAL, "null argument");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    const int nl = c->levels[c->depth].n;
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    if (!c->d_sflops) {
        float h[NSTREAM];
        for (int s = 0; s < NSTREAM; ++s) h[s] = (float)class_flops(s % NCLASS);
        KX_CUDA(c, cudaMalloc(&c->d_sflops, sizeof(h)));
        KX_CUDA(c, cudaMemcpy(c->d_sflops, h, sizeof(h), cudaMemcpyHostToDevice));
    }
    KX_TRY(grow(c, &c->d_work, &c->work_cap, (size_t)nl));
    KX_CUDA(c, cudaMemsetAsync(c->d_work, 0, sizeof(double) * nl, c->stream));
    kx_stats st;
    c->work_acc = c->d_work;
    const int r = kx_count(c, P, ldp, o, &st);
    c->work_acc = nullptr;
    if (r != KX_OK) return r;
    KX_CUDA(c, cudaMemcpyAsync(work, c->d_work, sizeof(double) * nl, cudaMemcpyDeviceToHost, c->stream));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    return KX_OK;
}

int kx_class_flops(int32_t cls, double* total, double* integral) {
    if (cls < 0 || cls >= NCLASS || !total || !integral) return KX_EINVAL;
    *total = class_flops(cls);
    *integral = integral_flops(class_l(cls));
    return KX_OK;
}

int kx_shard_bounds(const double* work, int32_t n_leaf, int32_t n_shards, int32_t* bounds) {
    if (!work || !bounds || n_leaf < 1 || n_shards < 1 || n_shards > n_leaf) return KX_EINVAL;
    double total = 0.0;
    for (int32_t i = 0; i < n_leaf; ++i) {
        if (!(work[i] >= 0.0) || !std::isfinite(work[i])) return KX_EINVAL;
        total += work[i];
    }
    std::vector<double> pre(n_leaf + 1, 0.0);   // pre[i] = work of leaves [0, i)
    for (int32_t i = 0; i < n_leaf; ++i) pre[i + 1] = pre[i] + (total > 0.0 ? work[i] : 1.0);
    const double all = pre[n_leaf];
    bounds[0] = 0;
    bounds[n_shards] = n_leaf;
    for (int32_t j = 1; j < n_shards; ++j) {
        // the leaf boundary whose prefix is nearest j/n of the total
        const double target = all * (double)j / (double)n_shards;
        int32_t i = (int32_t)(std::lower_bound(pre.begin(), pre.end(), target) - pre.begin());
        if (i > 0 && target - pre[i - 1] <= pre[std::min(i, n_leaf)] - target) --i;
        // every shard keeps at least one leaf
        i = std::max(i, bounds[j - 1] + 1);
        i = std::min(i, n_leaf - (n_shards - j));
        bounds[j] = i;
    }
    return KX_OK;
}

int kx_split_plan(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double budget, kx_stats* st) {
    KX_TRY(check_ctx(c));
    if (!P || !o || !st) return set_err(c, KX_EINVAL, "null argument");
    if (c->n_sys == 1 ? ldp < c->n_fn : true) return set_err(c, KX_EINVAL, "ldp must be >= n_fn");
    if (!std::isfinite(o->tau) || o->tau < 0.0) return set_err(c, KX_EINVAL, "tau must be >= 0");
    if (o->symmetric != 0 && o->symmetric != 1) return set_err(c, KX_EINVAL, "symmetric must be 0 or 1");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    std::memset(st, 0, sizeof(*st));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    return split_plan(c, P, ldp, o, budget, st);
}

int kx_exchange_batch(kx_ctx* c, const double* P, const kx_opts* o, double* K, kx_stats* st) {
    KX_TRY(check_ctx(c));
    return exchange_impl(c, P, 0, o, K, 0, st);
}

int kx_exchange_batch_host(kx_ctx* c, const double* P_host, const kx_opts* o, double* K_host, kx_stats* st) {
    KX_TRY(check_ctx(c));
    if (!P_host || !K_host || !o) return set_err(c, KX_EINVAL, "null argument");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    const size_t n = (size_t)c->sys_mat[c->n_sys];
    if (c->host_cap < n) {
        cudaFree(c->d_hostP);
        cudaFree(c->d_hostK);
        c->d_hostP = c->d_hostK = nullptr;
        c->host_cap = 0;
        KX_CUDA(c, cudaMalloc(&c->d_hostP, sizeof(double) * n));
        KX_CUDA(c, cudaMalloc(&c->d_hostK, sizeof(double) * n));
        c->host_cap = n;
    }
    KX_CUDA(c, cudaMemcpyAsync(c->d_hostP, P_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    KX_TRY(exchange_impl(c, c->d_hostP, 0, o, c->d_hostK, 0, st));
    KX_CUDA(c, cudaMemcpyAsync(K_host, c->d_hostK, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    return KX_OK;
}

int kx_autotune(kx_ctx* c, const double* P, const kx_opts* o, double* K, kx_stats* st, int32_t* n_tuned) {
    KX_TRY(check_ctx(c));
    if (!P || !K || !o) return set_err(c, KX_EINVAL, "null argument");
    if (!std::isfinite(o->tau) || o->tau < 0.0) return set_err(c, KX_EINVAL, "tau must be >= 0");
    if (o->precision < KX_FP64 || o->precision > KX_MIXED_DW) return set_err(c, KX_EINVAL, "bad precision");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    kx_stats local;
    kx_stats* s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    int n = 0;
    int r = autotune(c, P, o, K, s, &n);
    if (n_tuned) *n_tuned = n;
    return r;
}

int kx_get_launch_shapes(const kx_ctx* c, int32_t* threads, int32_t* blocks_per_sm, int32_t* variant) {
    if (!c) return KX_EINVAL;
    for (int s = 0; s < NSTREAM; ++s) {
        if (threads) threads[s] = c->eri_threads[s];
        if (blocks_per_sm) blocks_per_sm[s] = c->eri_bpsm[s];
        if (variant) variant[s] = c->eri_variant[s];
    }
    return KX_OK;
}

int kx_set_launch_shape(kx_ctx* c, int32_t s, int32_t threads, int32_t blocks_per_sm, int32_t variant) {
    KX_TRY(check_ctx(c));
    if (s < 0 || s >= NSTREAM || threads < 32 || threads > ERI_MAX_THREADS || threads % 32 || blocks_per_sm < 0)
        return set_err(c, KX_EINVAL, "bad launch shape");
    if (variant < 0 || variant >= eri_kernel(s % NCLASS, s / NCLASS, 0).n_variants)
        return set_err(c, KX_EINVAL, "no such kernel variant for this stream");
    drop_graph(c);
    c->eri_threads[s] = threads;
    c->eri_bpsm[s] = blocks_per_sm;
    c->eri_variant[s] = variant;
    return KX_OK;
}

int kx_graph_plan(kx_ctx* c, const double* P, const kx_opts* o, double* K, double headroom, kx_stats* st) {
    KX_TRY(check_ctx(c));
    if (!P || !K || !o) return set_err(c, KX_EINVAL, "null argument");
    if (!std::isfinite(o->tau) || o->tau < 0.0) return set_err(c, KX_EINVAL, "tau must be >= 0");
    if (o->precision < KX_FP64 || o->precision > KX_MIXED_DW) return set_err(c, KX_EINVAL, "bad precision");
    if (o->precision != KX_FP64 && (!std::isfinite(o->split_threshold) || o->split_threshold < 0.0))
        return set_err(c, KX_EINVAL, "split_threshold must be >= 0");
    if (!std::isfinite(headroom) || headroom < 0.0 || headroom > 16.0)
        return set_err(c, KX_EINVAL, "headroom must be in [0, 16]");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    if (!std::isfinite(o->split_budget) || o->split_budget < 0.0)
        return set_err(c, KX_EINVAL, "split_budget must be >= 0");
    kx_stats local;
    kx_stats* s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    // a split from the error budget is chosen once, for every replay
    kx_opts ob = *o;
    kx_stats sp;
    std::memset(&sp, 0, sizeof(sp));
    if (o->precision != KX_FP64 && o->split_budget > 0.0) {
        KX_TRY(split_plan(c, P, 0, o, o->split_budget, &sp));
        ob.split_threshold = sp.split_used;
        ob.split_budget = 0.0;
    }
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    const int r = graph_plan(c, P, &ob, K, headroom, s);
    c->graph_split = o->precision != KX_FP64 ? ob.split_threshold : 0.0;
    c->graph_err_est = sp.fp32_err_estimate;
    c->graph_err_bound = sp.fp32_err_bound;
    s->split_used = c->graph_split;
    s->fp32_err_estimate = c->graph_err_est;
    s->fp32_err_bound = c->graph_err_bound;
    return r;
}

int kx_graph_launch(kx_ctx* c, kx_stats* st) {
    KX_TRY(check_ctx(c));
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    return graph_launch(c, st);
}

int64_t kx_n_functions(const kx_ctx* c) { return c ? c->n_fn : -1; }

int64_t kx_packed_size(const kx_ctx* c) { return c ? c->sys_mat[c->n_sys] : -1; }

int kx_get_order(const kx_ctx* c, int32_t* perm) {
    if (!c || !perm) return KX_EINVAL;
    if (!c->have_order) return KX_ESTATE;
    std::memcpy(perm, c->perm.data(), sizeof(int32_t) * c->n_shell);
    return KX_OK;
}

int kx_get_leaves(const kx_ctx* c, int32_t* lo, int32_t* hi, int32_t cap, int32_t* n_leaf, int32_t* depth) {
    if (!c || !n_leaf || !depth) return KX_EINVAL;
    if (!c->have_tree) return KX_ESTATE;
    const int D = c->depth, nl = c->levels[D].n, off = c->levels[D].off;
    *n_leaf = nl;
    *depth = D;
    if (!lo || !hi) return KX_OK;
    if (cap < nl) return KX_ECAPACITY;
    std::memcpy(lo, c->node_lo.data() + off, sizeof(int32_t) * nl);
    std::memcpy(hi, c->node_hi.data() + off, sizeof(int32_t) * nl);
    return KX_OK;
}

int kx_get_worklist(kx_ctx* c, const int32_t* a_filter, int32_t n_filter, int32_t* out, int64_t cap, int64_t* n) {
    KX_TRY(check_ctx(c));
    if (!n || (n_filter > 0 && !a_filter) || n_filter < 0 || cap < 0 || (cap > 0 && !out))
        return set_err(c, KX_EINVAL, "bad argument");
    if (!c->keep_valid) return set_err(c, KX_ESTATE, "no worklist kept (set keep_worklist)");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    const int nl = c->levels[c->depth].n;
    uint8_t* d_mark = nullptr;
    Task* d_out = nullptr;
    unsigned long long* d_cnt = c->d_counters + CTR_FILTER;
    int r = KX_OK;
    cudaError_t e = cudaSuccess;
    if (n_filter > 0) {
        std::vector<uint8_t> mark(nl, 0);
        for (int i = 0; i < n_filter; ++i)
            if (a_filter[i] >= 0 && a_filter[i] < nl) mark[a_filter[i]] = 1;
        e = cudaMalloc(&d_mark, nl);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_mark, mark.data(), nl, cudaMemcpyHostToDevice, c->stream);
    }
    if (e == cudaSuccess && cap > 0) e = cudaMalloc(&d_out, sizeof(Task) * cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), c->stream);
    unsigned long long cnt = 0;
    if (n_filter == 0) {
        // the whole list, in kept order
        cnt = (unsigned long long)c->keep_n;
        const int64_t m = std::min<int64_t>((int64_t)cnt, cap);
        if (e == cudaSuccess && m > 0)
            e = cudaMemcpyAsync(d_out, c->d_keep, sizeof(Task) * m, cudaMemcpyDeviceToDevice, c->stream);
    } else if (e == cudaSuccess && c->keep_n > 0) {
        unsigned grid = (unsigned)std::min<size_t>((c->keep_n + 255) / 256, (size_t)c->n_sm * 32);
        k_filter_work<<<grid, 256, 0, c->stream>>>(c->d_keep, (int64_t)c->keep_n, d_mark, d_out, d_cnt, cap);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_filter > 0)
        e = cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) {
        *n = (int64_t)cnt;
        int64_t m = std::min<int64_t>((int64_t)cnt, cap);
        if (m > 0) {
            std::vector<Task> h(m);
            e = cudaMemcpy(h.data(), d_out, sizeof(Task) * m, cudaMemcpyDeviceToHost);
            for (int64_t i = 0; i < m; ++i) {
                out[4 * i] = h[i].a;
                out[4 * i + 1] = h[i].b;
                out[4 * i + 2] = h[i].c;
                out[4 * i + 3] = h[i].d;
            }
        }
        if (e == cudaSuccess && (int64_t)cnt > cap) r = set_err(c, KX_ECAPACITY, "worklist larger than cap");
    }
    if (e != cudaSuccess) r = cuda_check(c, e, "kx_get_worklist");
    cudaFree(d_mark);
    cudaFree(d_out);
    return r;
}

int kx_get_norms(kx_ctx* c, double* s2, double* pq) {
    KX_TRY(check_ctx(c));
    if (!c->have_schwarz) return set_err(c, KX_ESTATE, "kx_build_schwarz must come first");
    if (pq && !c->have_pq) return set_err(c, KX_ESTATE, "no P norms (run kx_exchange)");
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    // one dense block per system, in the system's user shell order
    std::vector<double> t((size_t)c->sp_total);
    const double* src[2] = {c->d_s2, c->d_pq};
    double* dst[2] = {s2, pq};
    for (int k = 0; k < 2; ++k) {
        if (!dst[k]) continue;
        KX_CUDA(c, cudaMemcpy(t.data(), src[k], sizeof(double) * t.size(), cudaMemcpyDeviceToHost));
        for (const Seg& g2 : c->sseg) {
            const int b = g2.base, n = g2.n;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j)
                    dst[k][g2.off + (size_t)(c->perm[b + i] - b) * n + (c->perm[b + j] - b)] =
                        t[g2.off + (size_t)i * n + j];
        }
    }
    return KX_OK;
}

int kx_get_profile(const kx_ctx* c, double* ms, int64_t* n, double* flops, int32_t* launches) {
    if (!c) return KX_EINVAL;
    for (int s = 0; s < NSTREAM; ++s) {
        if (ms) ms[s] = c->prof_ms[s];
        if (n) n[s] = c->prof_n[s];
        if (flops) flops[s] = c->prof_flops[s];
        if (launches) launches[s] = c->prof_launches[s];
    }
    return KX_OK;
}

int kx_peak_probe(int device, int precision, double* gflops) {
    if (!gflops || (precision != KX_FP64 && precision != KX_MIXED && precision != KX_PROBE_FP64_MMA &&
                    precision != KX_PROBE_DW))
        return KX_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        (void)cudaGetLastError();
        return KX_ECUDA;
    }
    DeviceGuard g(device);
    if (!g.ok) return KX_ECUDA;
    return peak_probe(device, precision, gflops);
}

const char* kx_last_error(const kx_ctx* c) { return c ? c->err.c_str() : "null context"; }

void kx_destroy(kx_ctx* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        if (g.ok) {
            cudaStreamSynchronize(c->stream);
            free_all(c);
        }
    }
    delete c;
}

}  // extern "C"
