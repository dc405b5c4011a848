// kx_noalloc.cu -- one traversal level (Eqs. 7, 8) without any allocation.
//
// kx_traverse_level_noalloc expands a caller-held frontier of level-k tasks
// into the level-(k+1) tasks whose bound exceeds tau, exactly like one step
// of the traversal inside kx_exchange, but it calls no cudaMalloc/cudaFree:
// its scratch (survivor masks, survivor counts, their offsets and the scan's
// tile sums) lives in the file-scope device array below, sized for frontiers
// of at most KX_NOALLOC_MAX_TASKS tasks.
//
// Host code cannot use the array's name as a device address (it is a
// host-side stand-in), so the first call on each device, with that device
// current, asks the runtime for the address with cudaGetSymbolAddress and
// caches it per device.  The children's bounds and the compaction are the
// device helpers of the traversal itself (kx_traverse_impl.cuh).
#include <algorithm>
#include <mutex>
#include <string>

#include "kx_traverse_impl.cuh"

namespace {

using kx::Task;
using kx::block_excl_scan64;

constexpr int64_t NA_MAX = KX_NOALLOC_MAX_TASKS;
constexpr int NA_T = 256, NA_I = 16, NA_TILE = NA_T * NA_I;
constexpr int64_t NA_TILES = (NA_MAX + NA_TILE - 1) / NA_TILE;   // 64

// scratch layout (bytes): counts | offsets | tile sums | tile offsets |
// total and bad-id count | masks
constexpr size_t OFF_CNT = 0;
constexpr size_t OFF_OFF = OFF_CNT + sizeof(int64_t) * NA_MAX;
constexpr size_t OFF_TSUM = OFF_OFF + sizeof(int64_t) * NA_MAX;
constexpr size_t OFF_TOFF = OFF_TSUM + sizeof(int64_t) * NA_TILES;
constexpr size_t OFF_TOTAL = OFF_TOFF + sizeof(int64_t) * NA_TILES;
constexpr size_t OFF_MASK = OFF_TOTAL + 256;
constexpr size_t NA_BYTES = OFF_MASK + sizeof(uint16_t) * NA_MAX;

static __device__ __align__(256) unsigned char kx_noalloc_scratch[NA_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[MAX_DEVICES] = {};

// device address of the scratch array on the current device (set up once)
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= MAX_DEVICES) return KX_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, kx_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return KX_ECUDA;
        }
        g_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[device];
    return KX_OK;
}

// children bounds of every task (the test of the traversal inside
// kx_exchange); a task naming a node id at or beyond the level's node count
// n_level gets no children and is counted in *bad, and none of its ids is
// used to index a table
__global__ void k_na_mask(const Task* __restrict__ front, int64_t n, int n_level, const int32_t* __restrict__ child,
                          const int32_t* __restrict__ nchild, const double* __restrict__ S,
                          const double* __restrict__ Pn, int nn, double tau, int sym, uint16_t* __restrict__ mask,
                          int64_t* __restrict__ cnt, unsigned long long* __restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Task t = front[i];
        unsigned m = 0;
        if (t.a < n_level && t.b < n_level && t.c < n_level && t.d < n_level)
            m = kx::task_child_mask(t, child, nchild, S, Pn, 0, nn, tau, sym && t.a == t.c, kx::RowRange{nullptr, nullptr, 0, 0});
        else
            atomicAdd(bad, 1ull);
        mask[i] = (uint16_t)m;
        cnt[i] = __popc(m);
    }
}

// per-tile sums of the counts
__global__ void __launch_bounds__(NA_T) k_na_tiles(const int64_t* __restrict__ cnt, int64_t n,
                                                   int64_t* __restrict__ tsum) {
    __shared__ int64_t sh[32];
    const int64_t base = blockIdx.x * (int64_t)NA_TILE + threadIdx.x * (int64_t)NA_I;
    int64_t s = 0;
    for (int k = 0; k < NA_I; ++k)
        if (base + k < n) s += cnt[base + k];
    int64_t total;
    block_excl_scan64(s, sh, &total);
    if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

// one block: exclusive scan of the (<= NA_TILES) tile sums and the grand total
__global__ void __launch_bounds__(NA_T) k_na_tile_scan(const int64_t* __restrict__ tsum, int ntiles,
                                                       int64_t* __restrict__ toff, int64_t* __restrict__ total) {
    __shared__ int64_t sh[32];
    const int64_t v = threadIdx.x < ntiles ? tsum[threadIdx.x] : 0;
    int64_t tot;
    const int64_t ex = block_excl_scan64(v, sh, &tot);
    if (threadIdx.x < ntiles) toff[threadIdx.x] = ex;
    if (threadIdx.x == 0) *total = tot;
}

// offsets of every task's first child
__global__ void __launch_bounds__(NA_T) k_na_offsets(const int64_t* __restrict__ cnt, int64_t n,
                                                     const int64_t* __restrict__ toff, int64_t* __restrict__ off) {
    __shared__ int64_t sh[32];
    const int64_t base = blockIdx.x * (int64_t)NA_TILE + threadIdx.x * (int64_t)NA_I;
    int64_t v[NA_I], s = 0;
    for (int k = 0; k < NA_I; ++k) {
        v[k] = base + k < n ? cnt[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t o = block_excl_scan64(s, sh, &total) + toff[blockIdx.x];
    for (int k = 0; k < NA_I; ++k) {
        if (base + k < n) off[base + k] = o;
        o += v[k];
    }
}

// children in the order (iA, iB, iC, iD); nothing is written at or past cap
// (a task without children -- culled or with a bad id -- reads no table)
__global__ void k_na_write(const Task* __restrict__ front, int64_t n, const uint16_t* __restrict__ mask,
                           const int64_t* __restrict__ off, const int32_t* __restrict__ child,
                           Task* __restrict__ out, int64_t cap) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned m = mask[i];
        if (!m) continue;
        kx::write_children(front[i], m, child, out, off[i], cap);
    }
}

struct Guard {
    int prev = -1;
    bool ok = true;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
        if (!ok) (void)cudaGetLastError();
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int kx_traverse_level_noalloc(kx_ctx* c, int32_t level, const uint16_t* front, int64_t n, double tau,
                                         uint16_t* next, int64_t cap, int64_t* n_next) {
    if (!c) return KX_EINVAL;
    if (c->n_sys != 1) return kx::set_err(c, KX_ENOTIMPL, "single-system contexts only");
    if (n > NA_MAX)
        return kx::set_err(c, KX_ECAPACITY, "frontier of " + std::to_string(n) + " tasks exceeds the " +
                                                std::to_string(NA_MAX) + "-task limit of the no-allocation path");
    if (!n_next || n < 0 || cap < 0 || (n > 0 && !front) || (cap > 0 && !next) || !(tau >= 0.0) ||
        tau > 1.7976931348623157e308)
        return kx::set_err(c, KX_EINVAL, "bad argument");
    if (!c->have_tree || !c->have_pq)
        return kx::set_err(c, KX_ESTATE, "needs the tree and the P norms of a previous kx_exchange");
    if (level < 0 || level >= c->depth) return kx::set_err(c, KX_EINVAL, "level must be in [0, depth)");
    Guard g(c->device);
    if (!g.ok) return kx::set_err(c, KX_ECUDA, "cudaSetDevice failed");
    unsigned char* base = nullptr;
    int r = scratch_address(c->device, &base);
    if (r != KX_OK) return kx::set_err(c, r, "cudaGetSymbolAddress of the scratch array failed");
    int64_t* cnt = reinterpret_cast<int64_t*>(base + OFF_CNT);
    int64_t* off = reinterpret_cast<int64_t*>(base + OFF_OFF);
    int64_t* tsum = reinterpret_cast<int64_t*>(base + OFF_TSUM);
    int64_t* toff = reinterpret_cast<int64_t*>(base + OFF_TOFF);
    int64_t* total = reinterpret_cast<int64_t*>(base + OFF_TOTAL);
    uint16_t* mask = reinterpret_cast<uint16_t*>(base + OFF_MASK);
    cudaStream_t st = c->stream;
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(base + OFF_TOTAL + 8);
    // the grand total (for an empty frontier) and the bad-id count start at zero
    cudaError_t e = cudaMemsetAsync(total, 0, 16, st);
    if (e == cudaSuccess && n > 0) {
        const int nn = c->levels[level + 1].n;
        const int n_level = c->levels[level].n;
        const int32_t* child = c->d_node_child + c->levels[level].off;
        const int32_t* nchild = c->d_node_nchild + c->levels[level].off;
        const double* S = c->d_nrm_s + c->pyr_off[level + 1];
        const double* Pn = c->d_nrm_p + c->pyr_off[level + 1];
        const Task* fr = reinterpret_cast<const Task*>(front);
        const unsigned g1 = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->n_sm * 16);
        const int ntiles = (int)((n + NA_TILE - 1) / NA_TILE);
        k_na_mask<<<g1, 256, 0, st>>>(fr, n, n_level, child, nchild, S, Pn, nn, tau, c->build_sym, mask, cnt, bad);
        k_na_tiles<<<ntiles, NA_T, 0, st>>>(cnt, n, tsum);
        k_na_tile_scan<<<1, NA_T, 0, st>>>(tsum, ntiles, toff, total);
        k_na_offsets<<<ntiles, NA_T, 0, st>>>(cnt, n, toff, off);
        k_na_write<<<g1, 256, 0, st>>>(fr, n, mask, off, child, reinterpret_cast<Task*>(next), cap);
        e = cudaGetLastError();
    }
    int64_t h[2] = {0, 0};   // total, bad ids
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, total, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return kx::cuda_check(c, e, "kx_traverse_level_noalloc");
    *n_next = h[0];
    if (h[1] != 0)
        return kx::set_err(c, KX_EINVAL, std::to_string(h[1]) + " tasks name node ids outside level " +
                                             std::to_string(level));
    if (h[0] > cap) return kx::set_err(c, KX_ECAPACITY, "next frontier larger than cap");
    return KX_OK;
}
