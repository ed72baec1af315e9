// Serving: many concurrent runs of Algorithm 1 (arXiv:1106.4198), one per
// stream, fed chunk by chunk; every chunk is one minibatch of its stream.
//
// Device side (onmf_serve.cuh): a batch of chunks of different streams,
// dictionary sizes and lengths runs as three phases, each one launch over
// all (chunk, work unit) pairs so even one chunk spreads over the GPU: the
// h-solve of every 8-frame tile (one launch over every dictionary size: the
// mma h-solve reads each chunk's size at run time), the statistics and W'
// of every (16 x 32) output tile, and the column rescale with the chunk's
// loss. Every (chunk, work unit) pair is computed in a fixed order of
// operations, so a chunk's result does not depend on the batch it runs in.
//
// Host side: onmf_server_submit copies a chunk's frames once, into a buffer
// of a pinned host arena mapped into the device's address space. A worker
// thread forms batches from the queued chunks of admitted streams that have
// nothing in flight (oldest chunk first), copies the batch's item table and
// a header of its layout to the device and launches, on one of `slots` CUDA
// streams, the gather of the frames from the arena and the three phases, by
// default as one CUDA graph captured once per slot (the kernels read the
// layout from the header, so the graph serves every batch unchanged); it records an event, and completed batches
// give their arena buffers back and are turned into completion records with
// submit/done timestamps. Stream states live in a device pool of
// budget_bytes reserved at creation (first-fit free list); a stream that
// does not fit waits in FIFO order until others close.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "onmf.h"
#include "onmf_launch.h"
#include "onmf_serve.cuh"

namespace onmf {

static size_t serve_smem(int F, int prec) {
    const Shape worst = make_shape(F, 128);
    return online_smem_bytes(worst, prec);
}

}  // namespace onmf

// =============================================================== runtime

using namespace onmf;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// First-fit allocator over one device pool (the serving budget).
struct Pool {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    size_t used = 0;
    void init(char *b, size_t n) {
        base = b;
        size = n;
        free_.clear();
        free_[0] = n;
        used = 0;
    }
    static size_t up(size_t x) { return (x + 255) / 256 * 256; }
    char *alloc(size_t n) {
        n = up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                used += n;
                return base + off;
            }
        }
        return nullptr;
    }
    void release(char *p, size_t n) {
        n = up(n);
        size_t off = p - base;
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// Pinned host memory for queued chunks, mapped into the device's address
// space so that a batch's first kernel reads the frames from it: size
// classes of 8 << c frames (c = 0..9), each a free list of buffers carved
// from slabs of at least 8 MB that live until the server is destroyed.
struct HostBuf {
    float *h = nullptr;        // host address
    const float *d = nullptr;  // device address of the same memory
    int cls = 0;
};

struct HostArena {
    static constexpr int kClasses = 10;
    int F = 1;
    std::mutex mu;
    std::vector<HostBuf> free_[kClasses];
    std::vector<void *> slabs;
    static int class_of(int n) {
        int c = 0;
        while ((8 << c) < n) ++c;
        return c;
    }
    size_t buf_bytes(int c) const { return ((size_t)(8 << c) * F * 4 + 255) / 256 * 256; }
    bool get(int n, HostBuf &b) {
        const int c = class_of(n);
        std::lock_guard<std::mutex> lk(mu);
        if (free_[c].empty()) {
            const size_t bb = buf_bytes(c), count = std::max<size_t>(1, (size_t(8) << 20) / bb);
            void *h = nullptr, *d = nullptr;
            if (cudaHostAlloc(&h, bb * count, cudaHostAllocMapped | cudaHostAllocPortable) !=
                cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
                cudaGetLastError();
                cudaFreeHost(h);
                return false;
            }
            slabs.push_back(h);
            for (size_t i = 0; i < count; ++i)
                free_[c].push_back(HostBuf{reinterpret_cast<float *>((char *)h + i * bb),
                                           reinterpret_cast<const float *>((char *)d + i * bb), c});
        }
        b = free_[c].back();
        free_[c].pop_back();
        return true;
    }
    void put(const HostBuf &b) {
        std::lock_guard<std::mutex> lk(mu);
        free_[b.cls].push_back(b);
    }
    ~HostArena() {
        for (void *h : slabs) cudaFreeHost(h);
    }
};

// A buffer of the arena, given back when destroyed.
struct Frames {
    HostArena *a = nullptr;
    HostBuf b;
    Frames() = default;
    Frames(HostArena *a_, const HostBuf &b_) : a(a_), b(b_) {}
    Frames(Frames &&o) noexcept : a(o.a), b(o.b) { o.a = nullptr; }
    Frames &operator=(Frames &&o) noexcept {
        if (this != &o) {
            reset();
            a = o.a;
            b = o.b;
            o.a = nullptr;
        }
        return *this;
    }
    Frames(const Frames &) = delete;
    Frames &operator=(const Frames &) = delete;
    ~Frames() { reset(); }
    void reset() {
        if (a) a->put(b);
        a = nullptr;
    }
};

struct Chunk {
    int64_t tag;
    int n;
    Frames v;  // F x n frames
    float *H_host;
    double t_submit;
};

struct StreamRec {
    int64_t id;
    onmf_config cfg;
    Shape s;
    std::vector<float> W0;
    size_t bytes = 0;
    char *mem = nullptr;
    float *Wcm = nullptr, *Wrm = nullptr, *Wn = nullptr, *swpart = nullptr;
    __nv_bfloat16 *Wimg = nullptr;
    double *A = nullptr, *B = nullptr, *loss_sum = nullptr;
    bool admitted = false, in_flight = false, closing = false, failed = false;
    std::deque<Chunk> queue;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr, ev0 = nullptr;  // end and start of the batch on the device
    cudaStream_t sub[8] = {};      // one per k16-slab count, joined back into `stream`
    cudaEvent_t ev_fork = nullptr, ev_join[8] = {};
    bool busy = false;
    ServeItem *d_items = nullptr, *h_items = nullptr;
    // batch header (hdr_ints(max_batch) ints, fixed layout): the work
    // offsets of the phases (tiles, units, columns, gather blocks;
    // max_batch + 1 each), then item ranges: [0, n) and one per k16-slab
    // count 1..8
    int *d_off = nullptr, *h_off = nullptr;
    // captured phase graphs by the set of k16-slab counts present (bit ks-1;
    // 0 on the FP32 path), with the number of kernels in each
    std::map<unsigned, std::pair<cudaGraphExec_t, int>> graphs;
    float *d_V = nullptr;  // the batch's frames, each chunk's slice 16-byte aligned
    float *d_H = nullptr, *h_H = nullptr;
    char *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    double *d_loss = nullptr, *h_loss = nullptr;
    int *d_err = nullptr, *h_err = nullptr;
    struct Done {
        int64_t stream, tag;
        int n;
        double t_submit;
        float *H_host;
        size_t h_off;
        int K;
        Frames v;  // held until the batch is done
    };
    std::vector<Done> chunks;
};

}  // namespace

struct onmf_server {
    onmf_server_config cfg;
    HostArena arena;  // declared before the slots and streams that hold its buffers
    int prec;
    // mixed path: one h-solve launch over every dictionary size of a batch
    // (default), or one launch per size on forked streams (ONMF_SERVE_FORK=1)
    bool fork_sizes = false;
    int nsm = 1;
    size_t smem = 0;
    size_t cap_frames = 0;
    Pool pool;
    char *pool_mem = nullptr;
    std::vector<Slot> slots;
    std::unordered_map<int64_t, StreamRec> streams;
    std::deque<int64_t> pending;   // streams waiting for memory
    std::deque<int64_t> arrivals;  // one entry per queued chunk, arrival order
    std::deque<onmf_completion> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1;
    onmf_server_stats st{};
    cudaStream_t admin = nullptr;
};

static size_t stream_bytes(const onmf_server *sv, const Shape &s) {
    const size_t FK = (size_t)s.F * s.K;
    size_t b = Pool::up(FK * 4) * 2 + Pool::up(FK * 8) * 2 + Pool::up((size_t)s.K * 4) + 256;
    if (sv->prec == PREC_FP32)
        b += Pool::up(FK * 4);
    else
        b += Pool::up((size_t)s.Kp * s.WLD * 2);
    return b;
}

// Carve the stream's state from the pool and initialize it (W0, zero A, B,
// loss, derived images). Caller holds the lock.
static bool admit(onmf_server *sv, StreamRec &r) {
    char *m = sv->pool.alloc(r.bytes);
    if (!m) return false;
    r.mem = m;
    const Shape &s = r.s;
    const size_t FK = (size_t)s.F * s.K;
    char *p = m;
    auto take = [&](size_t n) {
        char *q = p;
        p += Pool::up(n);
        return q;
    };
    r.Wcm = reinterpret_cast<float *>(take(FK * 4));
    r.Wn = reinterpret_cast<float *>(take(FK * 4));
    r.A = reinterpret_cast<double *>(take(FK * 8));
    r.B = reinterpret_cast<double *>(take(FK * 8));
    r.swpart = reinterpret_cast<float *>(take((size_t)s.K * 4));
    r.loss_sum = reinterpret_cast<double *>(take(256));
    if (sv->prec == PREC_FP32)
        r.Wrm = reinterpret_cast<float *>(take(FK * 4));
    else
        r.Wimg = reinterpret_cast<__nv_bfloat16 *>(take((size_t)s.Kp * s.WLD * 2));
    cudaStream_t q = sv->admin;
    bool ok = cudaMemcpyAsync(r.Wcm, r.W0.data(), FK * 4, cudaMemcpyHostToDevice, q) == cudaSuccess &&
              cudaMemsetAsync(r.A, 0, FK * 8, q) == cudaSuccess &&
              cudaMemsetAsync(r.B, 0, FK * 8, q) == cudaSuccess &&
              cudaMemsetAsync(r.loss_sum, 0, 8, q) == cudaSuccess;
    if (ok && r.Wimg) ok = cudaMemsetAsync(r.Wimg, 0, (size_t)s.Kp * s.WLD * 2, q) == cudaSuccess;
    if (ok) ok = launch_prepare(s, r.Wcm, r.Wrm, r.Wimg, r.swpart, q) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(q) == cudaSuccess;
    if (!ok) r.failed = true;
    r.admitted = true;
    sv->st.streams_admitted++;
    return true;
}

static void admit_pending(onmf_server *sv) {
    while (!sv->pending.empty()) {
        auto it = sv->streams.find(sv->pending.front());
        if (it == sv->streams.end()) {
            sv->pending.pop_front();
            continue;
        }
        if (!admit(sv, it->second)) break;
        sv->pending.pop_front();
    }
    sv->st.streams_pending = (int64_t)sv->pending.size();
    sv->st.bytes_in_use = (int64_t)sv->pool.used;
}

static void release_stream(onmf_server *sv, int64_t id) {
    auto it = sv->streams.find(id);
    if (it == sv->streams.end()) return;
    if (it->second.mem) sv->pool.release(it->second.mem, it->second.bytes);
    sv->streams.erase(it);
    admit_pending(sv);
}

// Form and launch one batch on a free slot. Returns true if launched.
static bool launch_batch_(onmf_server *sv, Slot &sl, std::unique_lock<std::mutex> &lk);

static int hdr_ints(int max_batch) { return 4 * (max_batch + 1) + 2 * 9; }

// The phases of one batch on the slot's stream, reading the batch's layout
// from the header in device memory. work[0..8] are the tiles per k16-slab
// count (work[0]: the FP32 path), work[9] the statistics units, work[10]
// the columns, work[11] the gather blocks. `fixed` gives every launch its largest grid (grid-stride
// loops take any work size), as a captured graph that serves every batch
// with the same set `mask` of slab counts needs; otherwise each grid is cut
// to its work.
static bool enqueue_phases(onmf_server *sv, Slot &sl, unsigned mask, const int *work, bool fixed,
                           int &nlaunch) {
    cudaStream_t q = sl.stream;
    const int nsm = sv->nsm, M1 = sv->cfg.max_batch + 1;
    const int *dt = sl.d_off, *du = dt + M1, *dc = du + M1, *dg = dc + M1, *dr = dg + M1;
    auto grid = [&](int w, int cap) { return fixed ? cap : std::min(w, cap); };
    auto launch = [&](const void *fn, int g, size_t smem, cudaStream_t st, const int *off,
                      const int *range) {
        const ServeItem *items = sl.d_items;
        void *args[] = {&items, &off, &range};
        ++nlaunch;
        return cudaLaunchKernel(fn, dim3(g), dim3(kThreads), args, smem, st) == cudaSuccess;
    };
    bool ok = cudaMemsetAsync(sl.d_err, 0, sizeof(int), q) == cudaSuccess;
    // phase 0: the frames from mapped host memory to the device
    if (ok) ok = launch(serve_gather_fn(), grid(work[11], 4 * nsm), 0, q, dg, dr);
    // phase 1: the h-solve, one launch over every chunk (the mixed kernel
    // reads each chunk's dictionary size at run time); with fork_sizes, one
    // launch per dictionary size (kernels specialized by size) on its own
    // stream, then join
    if (ok && (sv->prec == PREC_FP32 || !sv->fork_sizes)) {
        ok = launch(sv->prec == PREC_FP32 ? serve_fn(PREC_FP32, 0) : serve_any_fn(),
                    grid(work[0], nsm), sv->smem, q, dt, dr);
    } else if (ok) {
        ok = cudaEventRecord(sl.ev_fork, q) == cudaSuccess;
        for (int ks = 1; ok && ks <= 8; ++ks) {
            if (!((mask >> (ks - 1)) & 1u)) continue;
            cudaStream_t qs = sl.sub[ks - 1];
            ok = cudaStreamWaitEvent(qs, sl.ev_fork, 0) == cudaSuccess &&
                 launch(serve_fn(PREC_MIXED, ks), grid(work[ks], nsm), sv->smem, qs, dt,
                        dr + 2 * ks) &&
                 cudaEventRecord(sl.ev_join[ks - 1], qs) == cudaSuccess &&
                 cudaStreamWaitEvent(q, sl.ev_join[ks - 1], 0) == cudaSuccess;
        }
    }
    // phases 2 and 3 over every item of the batch
    if (ok)
        ok = launch(serve_stats_fn(sv->prec), grid(work[9], nsm), stats_smem_bytes(sv->prec), q,
                    du, dr);
    if (ok) ok = launch(serve_rescale_fn(sv->prec), grid(work[10], 4 * nsm), 0, q, dc, dr);
    return ok;
}

// Launches the phases as the slot's graph for `mask`, capturing and
// instantiating it on first use.
static bool launch_graph(onmf_server *sv, Slot &sl, unsigned mask, int &nlaunch) {
    auto it = sl.graphs.find(mask);
    if (it == sl.graphs.end()) {
        cudaStream_t q = sl.stream;
        int kernels = 0;
        if (cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
        const int none[12] = {};
        const bool queued = enqueue_phases(sv, sl, mask, none, true, kernels);
        cudaGraph_t g = nullptr;
        const bool ended = cudaStreamEndCapture(q, &g) == cudaSuccess;
        cudaGraphExec_t ex = nullptr;
        const bool ok = queued && ended && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            cudaGetLastError();
            return false;
        }
        it = sl.graphs.emplace(mask, std::make_pair(ex, kernels)).first;
    }
    nlaunch += it->second.second;
    return cudaGraphLaunch(it->second.first, sl.stream) == cudaSuccess;
}

static bool launch_batch(onmf_server *sv, Slot &sl, std::unique_lock<std::mutex> &lk) {
    nvtxRangePushA("serve batch");
    const bool r = launch_batch_(sv, sl, lk);
    nvtxRangePop();
    return r;
}

static bool launch_batch_(onmf_server *sv, Slot &sl, std::unique_lock<std::mutex> &lk) {
    const int F = sv->cfg.F;
    std::vector<std::pair<int64_t, Chunk>> picked;
    size_t frames = 0;
    for (auto it = sv->arrivals.begin(); it != sv->arrivals.end() &&
                                         (int)picked.size() < sv->cfg.max_batch;) {
        auto sit = sv->streams.find(*it);
        if (sit == sv->streams.end()) {
            it = sv->arrivals.erase(it);
            continue;
        }
        StreamRec &r = sit->second;
        bool taken = false;
        for (auto &pp : picked)
            if (pp.first == r.id) taken = true;
        if (!r.admitted || r.in_flight || taken || r.queue.empty()) {
            ++it;
            continue;
        }
        const size_t padded = (r.queue.front().n + 3) & ~3;
        if (frames + padded > sv->cap_frames) break;
        frames += padded;
        picked.emplace_back(r.id, std::move(r.queue.front()));
        r.queue.pop_front();
        r.in_flight = true;
        it = sv->arrivals.erase(it);
    }
    if (picked.empty()) return false;
    // snapshot the stream states used by this batch (pointers are stable while in flight)
    std::vector<StreamRec *> recs;
    for (auto &pp : picked) recs.push_back(&sv->streams[pp.first]);
    lk.unlock();
    // order the items by dictionary size: one launch per size
    {
        std::vector<size_t> ord(picked.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](size_t a, size_t b) { return recs[a]->s.Kp < recs[b]->s.Kp; });
        std::vector<std::pair<int64_t, Chunk>> p2;
        std::vector<StreamRec *> r2;
        for (size_t i : ord) {
            p2.push_back(std::move(picked[i]));
            r2.push_back(recs[i]);
        }
        picked.swap(p2);
        recs.swap(r2);
    }
    sl.chunks.clear();
    const auto t_form = std::chrono::steady_clock::now();
    size_t voff = 0, hoff = 0, soff = 0;
    const int elem = sv->prec == PREC_FP32 ? 4 : 2;
    for (size_t i = 0; i < picked.size(); ++i) {
        Chunk &c = picked[i].second;
        StreamRec &r = *recs[i];
        const Shape &s = r.s;
        const int betap = (c.n + 15) / 16 * 16;
        ServeItem it;
        memset(&it, 0, sizeof it);
        it.s = s;
        it.n = c.n;
        it.n_in = r.cfg.n_inner;
        it.eps = (float)r.cfg.eps;
        it.gamma = (float)r.cfg.h_exponent;
        it.normalize = r.cfg.normalize;
        it.rho_on_new = r.cfg.rho_on_new;
        it.rho = r.cfg.n_ref > 0 ? std::pow(r.cfg.r, (double)c.n / (double)r.cfg.n_ref) : 1.0;
        it.V = sl.d_V + voff * F;  // voff is a multiple of 4 frames: 16-byte aligned
        it.Vsrc = c.v.b.d;
        it.H_out = c.H_host ? sl.d_H + hoff : nullptr;
        it.Wcm = r.Wcm;
        it.Wrm = r.Wrm;
        it.Wn = r.Wn;
        it.swpart = r.swpart;
        it.Wimg = r.Wimg;
        it.A = r.A;
        it.B = r.B;
        it.loss_sum = r.loss_sum;
        // item scratch: P, Q (betap x Fp16), H (betap x Kh), loss slots
        char *sc = sl.d_scratch + soff;
        const size_t pq = Pool::up((size_t)betap * s.Fp16 * elem);
        const size_t hg = Pool::up((size_t)betap * s.Kh * elem);
        const size_t lp = Pool::up((size_t)((c.n + kTile - 1) / kTile) * 8);
        it.Pg = sc;
        it.Qg = sc + pq;
        it.Hg = sc + 2 * pq;
        it.loss_part = reinterpret_cast<double *>(sc + 2 * pq + hg);
        soff += 2 * pq + hg + lp;
        it.betap = betap;
        it.chunk_loss = sl.d_loss + i;
        it.err = sl.d_err;
        sl.h_items[i] = it;
        sl.chunks.push_back(
            {picked[i].first, c.tag, c.n, c.t_submit, c.H_host, hoff, s.K, std::move(c.v)});
        voff += (c.n + 3) & ~3;
        if (c.H_host) hoff += (size_t)c.n * s.K;
    }
    const int n = (int)picked.size();
    cudaStream_t q = sl.stream;
    // the batch header: work offsets of the three phases (8-frame tiles,
    // (16 x 32) output tiles, columns + the loss) and the item ranges
    const int M1 = sv->cfg.max_batch + 1;
    int *t_off = sl.h_off, *u_off = t_off + M1, *c_off = u_off + M1, *g_off = c_off + M1;
    int *rng = g_off + M1;
    t_off[0] = u_off[0] = c_off[0] = g_off[0] = 0;
    for (int i = 0; i < n; ++i) {
        const Shape &s = recs[i]->s;
        t_off[i + 1] = t_off[i] + ceil_div(sl.h_items[i].n, kTile);
        u_off[i + 1] = u_off[i] + (s.Fp16 / 16) * (s.Kh / 32);
        c_off[i + 1] = c_off[i] + s.K + 1;
        const long long f4 = ((long long)sl.h_items[i].n * F + 3) / 4;
        g_off[i + 1] = g_off[i] + (int)((f4 + kGatherF4 - 1) / kGatherF4);
    }
    rng[0] = 0;
    rng[1] = n;
    int work[12] = {};
    work[0] = t_off[n];
    work[9] = u_off[n];
    work[10] = c_off[n];
    work[11] = g_off[n];
    unsigned mask = 0;
    if (sv->prec != PREC_FP32) {
        for (int i0 = 0; i0 < n;) {
            const int ks = recs[i0]->s.Kp / 16;
            int i1 = i0;
            while (i1 < n && recs[i1]->s.Kp / 16 == ks) ++i1;
            rng[2 * ks] = i0;
            rng[2 * ks + 1] = i1;
            work[ks] = t_off[i1] - t_off[i0];
            mask |= 1u << (ks - 1);
            i0 = i1;
        }
    }
    bool ok = soff <= sl.scratch_bytes;
    if (ok) ok = cudaEventRecord(sl.ev0, q) == cudaSuccess;
    if (ok) ok = cudaMemcpyAsync(sl.d_items, sl.h_items, n * sizeof(ServeItem), cudaMemcpyHostToDevice, q) == cudaSuccess;
    if (ok)
        ok = cudaMemcpyAsync(sl.d_off, sl.h_off, hdr_ints(sv->cfg.max_batch) * sizeof(int),
                             cudaMemcpyHostToDevice, q) == cudaSuccess;
    const int64_t form_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(
                                std::chrono::steady_clock::now() - t_form).count();
    int nlaunch = 0;
    // one graph serves every batch unless the h-solve forks by size
    const unsigned gkey = sv->fork_sizes ? mask : 0u;
    if (ok)
        ok = sv->cfg.launch == ONMF_SERVE_GRAPH ? launch_graph(sv, sl, gkey, nlaunch)
                                                : enqueue_phases(sv, sl, mask, work, false, nlaunch);
    if (ok) ok = cudaMemcpyAsync(sl.h_loss, sl.d_loss, n * 8, cudaMemcpyDeviceToHost, q) == cudaSuccess;
    if (ok && hoff) ok = cudaMemcpyAsync(sl.h_H, sl.d_H, hoff * 4, cudaMemcpyDeviceToHost, q) == cudaSuccess;
    if (ok) ok = cudaMemcpyAsync(sl.h_err, sl.d_err, 4, cudaMemcpyDeviceToHost, q) == cudaSuccess;
    if (ok) ok = cudaEventRecord(sl.ev, q) == cudaSuccess;
    lk.lock();
    int busy_other = 0;
    for (auto &o : sv->slots)
        if (o.busy) ++busy_other;
    sl.busy = true;
    if (!ok) *sl.h_err = -1;
    sv->st.launches += nlaunch;
    sv->st.host_batch_ns += form_ns;
    if (busy_other) sv->st.batches_overlapped++;
    return true;
}

static void finish_batch(onmf_server *sv, Slot &sl) {
    const double t = now_s();
    const int err = *sl.h_err;
    float ms = 0.f;
    if (err == 0 && cudaEventElapsedTime(&ms, sl.ev0, sl.ev) == cudaSuccess)
        sv->st.device_ns += (int64_t)(1e6 * ms);
    for (size_t i = 0; i < sl.chunks.size(); ++i) {
        auto &c = sl.chunks[i];
        onmf_completion cp;
        memset(&cp, 0, sizeof cp);
        cp.stream_id = c.stream;
        cp.tag = c.tag;
        cp.frames = c.n;
        cp.loss = sl.h_loss[i];
        cp.t_submit = c.t_submit;
        cp.t_done = t;
        cp.status = err == 0 ? ONMF_OK : (err < 0 ? ONMF_ECUDA : ONMF_ENUMERIC);
        if (c.H_host) memcpy(c.H_host, sl.h_H + c.h_off, (size_t)c.n * c.K * 4);
        c.v.reset();  // the frames have been read: the buffer goes back to the arena
        sv->done.push_back(cp);
        sv->st.chunks++;
        sv->st.frames += c.n;
        auto it = sv->streams.find(c.stream);
        if (it != sv->streams.end()) {
            StreamRec &r = it->second;
            r.in_flight = false;
            if (err) r.failed = true;
            if (r.closing && r.queue.empty()) release_stream(sv, c.stream);
        }
    }
    sl.busy = false;
}

static void worker_main(onmf_server *sv) {
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool progressed = false;
        for (auto &sl : sv->slots) {
            if (sl.busy && cudaEventQuery(sl.ev) == cudaSuccess) {
                finish_batch(sv, sl);
                progressed = true;
            }
        }
        if (progressed) {
            sv->cv_done.notify_all();
            sv->cv_work.notify_all();
        }
        for (auto &sl : sv->slots) {
            if (!sl.busy && launch_batch(sv, sl, lk)) progressed = true;
        }
        bool busy = false;
        for (auto &sl : sv->slots) busy |= sl.busy;
        if (sv->stop && !busy && sv->arrivals.empty()) break;
        if (!progressed) {
            if (busy)
                sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

static void free_server(onmf_server *sv) {
    for (auto &sl : sv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        for (auto &g : sl.graphs) cudaGraphExecDestroy(g.second.first);
        void *dev[] = {sl.d_items, sl.d_off, sl.d_V, sl.d_H, sl.d_scratch, sl.d_loss, sl.d_err};
        for (void *p : dev)
            if (p) cudaFree(p);
        void *host[] = {sl.h_items, sl.h_off, sl.h_H, sl.h_loss, sl.h_err};
        for (void *p : host)
            if (p) cudaFreeHost(p);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.ev0) cudaEventDestroy(sl.ev0);
        if (sl.ev_fork) cudaEventDestroy(sl.ev_fork);
        for (int g = 0; g < 8; ++g) {
            if (sl.ev_join[g]) cudaEventDestroy(sl.ev_join[g]);
            if (sl.sub[g]) cudaStreamDestroy(sl.sub[g]);
        }
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (sv->pool_mem) cudaFree(sv->pool_mem);
    if (sv->admin) cudaStreamDestroy(sv->admin);
    delete sv;
}

extern "C" {

onmf_status onmf_server_create(const onmf_server_config *cfg, onmf_server **out) {
    if (!cfg || !out) return ONMF_EINVAL;
    *out = nullptr;
    const onmf_server_config &c = *cfg;
    if (c.F < 1 || c.F > 1024 || c.max_chunk < 1 || c.max_chunk > 4096 || c.max_batch < 1 ||
        c.max_batch > 4096 || c.slots < 1 || c.slots > 4 || c.budget_bytes < 1 ||
        (c.launch != ONMF_SERVE_GRAPH && c.launch != ONMF_SERVE_DIRECT) ||
        (c.precision != ONMF_FP32 && c.precision != ONMF_MIXED))
        return ONMF_EINVAL;
    if (configure_kernels() != cudaSuccess) return ONMF_ECUDA;
    onmf_server *sv = new onmf_server();
    sv->cfg = c;
    sv->arena.F = c.F;
    sv->prec = c.precision == ONMF_MIXED ? PREC_MIXED : PREC_FP32;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sv->nsm, cudaDevAttrMultiProcessorCount, dev);
    sv->smem = serve_smem(c.F, sv->prec);
    {
        const char *fk = getenv("ONMF_SERVE_FORK");
        sv->fork_sizes = sv->prec != PREC_FP32 && fk && strcmp(fk, "1") == 0;
    }
    if (sv->smem > max_dynamic_smem()) {
        delete sv;
        return ONMF_EINVAL;
    }
    // frames per batch: enough for max_batch average chunks, at least one largest chunk
    // (chunk slices start at multiples of 4 frames)
    sv->cap_frames = std::max<size_t>(((size_t)c.max_chunk + 3) & ~size_t(3),
                                      std::min<size_t>((size_t)c.max_batch * 128, 65536));
    const Shape worst = make_shape(c.F, 128);
    const int elem = sv->prec == PREC_FP32 ? 4 : 2;
    const size_t per_frame = (size_t)worst.Fp16 * elem * 2 + (size_t)worst.Kh * elem + 8;
    if (cudaStreamCreateWithFlags(&sv->admin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void **)&sv->pool_mem, (size_t)c.budget_bytes) != cudaSuccess) {
        free_server(sv);
        return ONMF_ENOMEM;
    }
    sv->pool.init(sv->pool_mem, (size_t)c.budget_bytes);
    sv->slots.resize(c.slots);
    for (auto &sl : sv->slots) {
        sl.scratch_bytes = (sv->cap_frames + 16 * (size_t)c.max_batch) * per_frame + 1024 * (size_t)c.max_batch;
        bool ok =
            cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&sl.ev) == cudaSuccess && cudaEventCreate(&sl.ev0) == cudaSuccess &&
            cudaEventCreateWithFlags(&sl.ev_fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc((void **)&sl.d_items, c.max_batch * sizeof(ServeItem)) == cudaSuccess &&
            cudaHostAlloc((void **)&sl.h_items, c.max_batch * sizeof(ServeItem), 0) == cudaSuccess &&
            cudaMalloc((void **)&sl.d_off, hdr_ints(c.max_batch) * sizeof(int)) == cudaSuccess &&
            cudaHostAlloc((void **)&sl.h_off, hdr_ints(c.max_batch) * sizeof(int), 0) == cudaSuccess &&
            cudaMalloc((void **)&sl.d_V, sv->cap_frames * c.F * 4) == cudaSuccess &&
            cudaMalloc((void **)&sl.d_H, sv->cap_frames * 128 * 4) == cudaSuccess &&
            cudaHostAlloc((void **)&sl.h_H, sv->cap_frames * 128 * 4, 0) == cudaSuccess &&
            cudaMalloc((void **)&sl.d_scratch, sl.scratch_bytes) == cudaSuccess &&
            cudaMalloc((void **)&sl.d_loss, c.max_batch * 8) == cudaSuccess &&
            cudaHostAlloc((void **)&sl.h_loss, c.max_batch * 8, 0) == cudaSuccess &&
            cudaMalloc((void **)&sl.d_err, 16) == cudaSuccess &&
            cudaHostAlloc((void **)&sl.h_err, 16, 0) == cudaSuccess;
        for (int g = 0; ok && g < 8; ++g)
            ok = cudaStreamCreateWithFlags(&sl.sub[g], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.ev_join[g], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            free_server(sv);
            return ONMF_ENOMEM;
        }
        // zero scratch once: padded rows/columns of P, Q and H must read as zero
        if (cudaMemset(sl.d_scratch, 0, sl.scratch_bytes) != cudaSuccess) {
            free_server(sv);
            return ONMF_ECUDA;
        }
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return ONMF_OK;
}

onmf_status onmf_server_open_stream(onmf_server *sv, const onmf_config *cfg, const float *W0,
                                    int64_t *stream_id) {
    if (!sv || !cfg || !W0 || !stream_id) return ONMF_EINVAL;
    const onmf_config &c = *cfg;
    // serving runs the mma h-solve (AUTO or MMA) with FP64 statistics
    if (c.F != sv->cfg.F || c.K < 1 || c.K > 128 || c.n_inner < 0 || !(c.eps >= 0.0) ||
        !(c.h_exponent > 0.0) || !(c.r >= 0.0 && c.r <= 1.0) ||
        (c.hsolve != ONMF_HSOLVE_AUTO && c.hsolve != ONMF_HSOLVE_MMA) ||
        c.accumulate != ONMF_ACC_FP64 || c.stats_ranges < 0 || c.stats_ranges > kMaxRanges ||
        c.h_penalty != 0.0 || c.w_penalty != 0.0)
        return ONMF_EINVAL;
    StreamRec r;
    r.cfg = c;
    r.s = make_shape(c.F, c.K);
    r.W0.assign(W0, W0 + (size_t)c.F * c.K);
    for (float w : r.W0)
        if (!(w >= 0.f) || std::isinf(w)) return ONMF_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    r.bytes = stream_bytes(sv, r.s);
    if (r.bytes > (size_t)sv->cfg.budget_bytes) return ONMF_EBUDGET;
    r.id = sv->next_id++;
    *stream_id = r.id;
    auto &rec = sv->streams[r.id] = std::move(r);
    if (!sv->pending.empty() || !admit(sv, rec)) sv->pending.push_back(rec.id);
    sv->st.streams_pending = (int64_t)sv->pending.size();
    sv->st.bytes_in_use = (int64_t)sv->pool.used;
    return ONMF_OK;
}

onmf_status onmf_server_submit(onmf_server *sv, int64_t id, const float *V, int64_t ldv, int64_t n,
                               float *H_out, int64_t tag) {
    if (!sv || !V || n < 1 || n > sv->cfg.max_chunk || ldv < sv->cfg.F) return ONMF_EINVAL;
    Chunk c;
    c.tag = tag;
    c.n = (int)n;
    c.H_host = H_out;
    const int F = sv->cfg.F;
    HostBuf b;
    if (!sv->arena.get((int)n, b)) return ONMF_ENOMEM;
    c.v = Frames(&sv->arena, b);
    if (ldv == F)
        memcpy(b.h, V, (size_t)n * F * 4);
    else
        for (int64_t j = 0; j < n; ++j) memcpy(b.h + j * F, V + j * ldv, (size_t)F * 4);
    c.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->streams.find(id);
        if (it == sv->streams.end() || it->second.closing) return ONMF_EINVAL;
        if (it->second.failed) return ONMF_ESTATE;
        it->second.queue.push_back(std::move(c));
        sv->arrivals.push_back(id);
    }
    sv->cv_work.notify_one();
    return ONMF_OK;
}

onmf_status onmf_server_submit_many(onmf_server *sv, int32_t count, const int64_t *stream_ids,
                                    const float *const *V, const int64_t *ldv, const int64_t *n,
                                    float *const *H_out, const int64_t *tags, int32_t *queued) {
    if (queued) *queued = 0;
    if (!sv || count < 0 || (count > 0 && (!stream_ids || !V || !ldv || !n || !tags)))
        return ONMF_EINVAL;
    for (int32_t i = 0; i < count; ++i) {
        const onmf_status st = onmf_server_submit(sv, stream_ids[i], V[i], ldv[i], n[i],
                                                  H_out ? H_out[i] : nullptr, tags[i]);
        if (st != ONMF_OK) return st;
        if (queued) *queued = i + 1;
    }
    return ONMF_OK;
}

onmf_status onmf_server_poll(onmf_server *sv, onmf_completion *out, int32_t max, int32_t *count,
                             int32_t wait_ms) {
    if (!sv || !count || (max > 0 && !out)) return ONMF_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->done.empty() && wait_ms > 0)
        sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                             [&] { return !sv->done.empty(); });
    int k = 0;
    while (k < max && !sv->done.empty()) {
        out[k++] = sv->done.front();
        sv->done.pop_front();
    }
    *count = k;
    return ONMF_OK;
}

onmf_status onmf_server_get_W(onmf_server *sv, int64_t id, float *W_out) {
    if (!sv || !W_out) return ONMF_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        auto it = sv->streams.find(id);
        if (it == sv->streams.end()) return ONMF_EINVAL;
        StreamRec &r = it->second;
        if (r.admitted && !r.in_flight && r.queue.empty()) {
            const size_t FK = (size_t)r.s.F * r.s.K;
            cudaError_t e = cudaMemcpyAsync(W_out, r.Wcm, FK * 4, cudaMemcpyDeviceToHost, sv->admin);
            if (e == cudaSuccess) e = cudaStreamSynchronize(sv->admin);
            if (e != cudaSuccess) return ONMF_ECUDA;
            return r.failed ? ONMF_ESTATE : ONMF_OK;
        }
        sv->cv_done.wait_for(lk, std::chrono::milliseconds(10));
    }
}

onmf_status onmf_server_close_stream(onmf_server *sv, int64_t id) {
    if (!sv) return ONMF_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->streams.find(id);
    if (it == sv->streams.end()) return ONMF_EINVAL;
    StreamRec &r = it->second;
    r.closing = true;
    if (!r.admitted) {
        // never admitted: drop it (and its queued chunks) from the waiting line
        sv->pending.erase(std::remove(sv->pending.begin(), sv->pending.end(), id), sv->pending.end());
        sv->streams.erase(it);
        sv->st.streams_pending = (int64_t)sv->pending.size();
        return ONMF_OK;
    }
    if (!r.in_flight && r.queue.empty()) release_stream(sv, id);
    sv->cv_work.notify_one();
    return ONMF_OK;
}

onmf_status onmf_server_get_stats(onmf_server *sv, onmf_server_stats *out) {
    if (!sv || !out) return ONMF_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->st.streams_pending = (int64_t)sv->pending.size();
    sv->st.bytes_in_use = (int64_t)sv->pool.used;
    *out = sv->st;
    return ONMF_OK;
}

void onmf_server_destroy(onmf_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        // streams still waiting for memory would never run: drop their chunks
        for (int64_t id : sv->pending) {
            auto it = sv->streams.find(id);
            if (it != sv->streams.end()) it->second.queue.clear();
        }
        sv->arrivals.erase(std::remove_if(sv->arrivals.begin(), sv->arrivals.end(),
                                          [&](int64_t id) {
                                              auto it = sv->streams.find(id);
                                              return it == sv->streams.end() || !it->second.admitted;
                                          }),
                           sv->arrivals.end());
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    free_server(sv);
}

}  // extern "C"
