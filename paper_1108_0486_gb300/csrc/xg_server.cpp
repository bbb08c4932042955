// Request server: continuous batching of generation requests on resident
// streams.
//
//   submit  -> admission: outstanding output bytes (library pool and caller
//              buffers) stay under the memory cap, else XG_EAGAIN; a pool
//              buffer is carved when the caller passes no output.
//   queue   -> per-stream FIFO; a stream has at most one request on the GPU,
//              so its requests run in submission order.
//   batch   -> whenever a lane (CUDA stream with its own batch launcher) is
//              free, the oldest ready requests (one per stream) form a batch
//              that runs as one replay of the persistent batch kernel graph.
//              Batches on different lanes overlap on the device, so requests
//              that arrive while others run start as soon as a lane frees.
//   complete-> the kernel fences each request's stores and sets its flag in
//              mapped pinned host memory; xg_poll reads it directly.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "xg_batch.h"
#include "xg_jump.h"
#include "xg_runtime.h"

namespace xg {

static uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Sub-allocator over one device slab in O(1) per call: two-level segregated
// free lists (size classes of 16 per power of two, with bitmaps to find the
// smallest non-empty class that fits), blocks split on allocation and merged
// with free neighbours on release (physical neighbours are linked, so no
// search).  Block records live on the host; a request keeps its block's
// handle.  Sizes are in 256-byte units.
class DevicePool {
public:
    ~DevicePool()
    {
        if (base_) cudaFree(base_);
    }
    xg_status init(size_t cap)
    {
        cap_ = cap / kAlign * kAlign;
        if (cudaMalloc(reinterpret_cast<void**>(&base_), cap_) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return fail(XG_ENOMEM, "server pool: cudaMalloc(%zu) failed", cap_);
        }
        blk_.clear();
        spare_.clear();
        fl_map_ = 0;
        for (int f = 0; f < kFl; ++f) {
            sl_map_[f] = 0;
            for (int t = 0; t < kSl; ++t) heads_[f][t] = kNil;
        }
        const uint32_t b = new_block();
        blk_[b] = Block{0, cap_ / kAlign, kNil, kNil, kNil, kNil, true};
        insert_free(b);
        return XG_OK;
    }
    void* alloc(size_t bytes, uint32_t* handle)
    {
        const uint64_t u = std::max<uint64_t>(1, (bytes + kAlign - 1) / kAlign);
        const uint32_t b = find_fit(u);
        if (b == kNil) return nullptr;
        remove_free(b);
        if (blk_[b].units > u) {  // split off the rest as a free block
            const uint32_t r = new_block();
            Block& x = blk_[b];
            blk_[r] = Block{x.off + u, x.units - u, b, x.next_phys, kNil, kNil, true};
            if (x.next_phys != kNil) blk_[x.next_phys].prev_phys = r;
            x.next_phys = r;
            x.units = u;
            insert_free(r);
        }
        blk_[b].free = false;
        *handle = b;
        return base_ + blk_[b].off * kAlign;
    }
    void release(uint32_t b)
    {
        if (b >= blk_.size() || blk_[b].free) return;
        blk_[b].free = true;
        const uint32_t n = blk_[b].next_phys;
        if (n != kNil && blk_[n].free) {  // absorb the next block
            remove_free(n);
            blk_[b].units += blk_[n].units;
            blk_[b].next_phys = blk_[n].next_phys;
            if (blk_[n].next_phys != kNil) blk_[blk_[n].next_phys].prev_phys = b;
            spare_.push_back(n);
        }
        const uint32_t p = blk_[b].prev_phys;
        if (p != kNil && blk_[p].free) {  // be absorbed by the previous block
            remove_free(p);
            blk_[p].units += blk_[b].units;
            blk_[p].next_phys = blk_[b].next_phys;
            if (blk_[b].next_phys != kNil) blk_[blk_[b].next_phys].prev_phys = p;
            spare_.push_back(b);
            insert_free(p);
            return;
        }
        insert_free(b);
    }
    size_t capacity() const { return cap_; }

private:
    static constexpr size_t kAlign = 256;
    static constexpr int kSlBits = 4, kSl = 1 << kSlBits, kFl = 64;
    static constexpr uint32_t kNil = 0xFFFFFFFFu;
    struct Block {
        uint64_t off, units;           // in kAlign units
        uint32_t prev_phys, next_phys;  // neighbours in address order
        uint32_t prev_free, next_free;  // free list of its class
        bool free;
    };
    // Class of a size: sizes below 16 units exactly; above, 16 classes per
    // power of two.
    static void mapping(uint64_t u, int& f, int& t)
    {
        if (u < (uint64_t)kSl) {
            f = 0;
            t = (int)u;
            return;
        }
        const int msb = 63 - __builtin_clzll(u);
        f = msb - kSlBits + 1;
        t = (int)((u >> (msb - kSlBits)) & (kSl - 1));
    }
    uint32_t new_block()
    {
        if (!spare_.empty()) {
            const uint32_t b = spare_.back();
            spare_.pop_back();
            return b;
        }
        blk_.push_back(Block{});
        return (uint32_t)(blk_.size() - 1);
    }
    void insert_free(uint32_t b)
    {
        int f, t;
        mapping(blk_[b].units, f, t);
        blk_[b].prev_free = kNil;
        blk_[b].next_free = heads_[f][t];
        if (heads_[f][t] != kNil) blk_[heads_[f][t]].prev_free = b;
        heads_[f][t] = b;
        sl_map_[f] |= 1u << t;
        fl_map_ |= uint64_t(1) << f;
    }
    void remove_free(uint32_t b)
    {
        int f, t;
        mapping(blk_[b].units, f, t);
        const uint32_t p = blk_[b].prev_free, n = blk_[b].next_free;
        if (p != kNil) blk_[p].next_free = n;
        else heads_[f][t] = n;
        if (n != kNil) blk_[n].prev_free = p;
        if (heads_[f][t] == kNil) {
            sl_map_[f] &= ~(1u << t);
            if (!sl_map_[f]) fl_map_ &= ~(uint64_t(1) << f);
        }
    }
    // A free block of at least u units from the smallest class whose every
    // block fits (u rounded up to its class's upper bound), or kNil.
    uint32_t find_fit(uint64_t u) const
    {
        uint64_t r = u;
        if (u >= (uint64_t)kSl) r = u + (uint64_t(1) << (63 - __builtin_clzll(u) - kSlBits)) - 1;
        int f, t;
        mapping(r, f, t);
        uint32_t bits = f < kFl ? sl_map_[f] & (~0u << t) : 0u;
        if (!bits && f + 1 < kFl) {
            const uint64_t fb = fl_map_ & (~uint64_t(0) << (f + 1));
            if (fb) {
                f = __builtin_ctzll(fb);
                bits = sl_map_[f];
            }
        }
        if (bits) return heads_[f][__builtin_ctz(bits)];
        // no class is certain to fit: look through u's own class (its blocks
        // may still be large enough), a bounded first fit
        mapping(u, f, t);
        int seen = 0;
        for (uint32_t b = heads_[f][t]; b != kNil && seen < 256; b = blk_[b].next_free, ++seen)
            if (blk_[b].units >= u) return b;
        return kNil;
    }
    char* base_ = nullptr;
    size_t cap_ = 0;
    std::vector<Block> blk_;
    std::vector<uint32_t> spare_;
    uint32_t heads_[kFl][kSl];
    uint32_t sl_map_[kFl] = {};
    uint64_t fl_map_ = 0;
};

struct Ticket {
    uint64_t id = 0;
    uint64_t seq = 0;
    xg_request req{};
    void* out = nullptr;
    bool pooled = false;
    uint32_t pool_block = 0;  // the pool's handle of its output (when pooled)
    size_t bytes = 0;
    uint32_t slot = 0;
    uint32_t expected = 1;      // completion increments: 1, or the pieces it was cut into
    std::atomic<int> state{0};  // kQueued, kRunning, kDone, kFailed, kCancelled
    // who owns a queued request: 0 = nobody yet, 1 = the scheduler took it
    // into a batch, 2 = xg_cancel took it (the one that swaps it from 0 wins)
    std::atomic<int> claim{0};
    uint64_t t_submit = 0, t_launch = 0;
    std::atomic<uint64_t> t_done{0};
    std::shared_ptr<Ticket> next_in_stream;  // the stream's queue (scheduler thread only)
};

// A stream's queue of admitted requests (an intrusive list through the
// tickets, so queueing allocates nothing) and whether one of its requests
// is on the GPU.
struct StreamQueue {
    std::shared_ptr<Ticket> head;
    Ticket* tail = nullptr;
    bool busy = false;
    void push(const std::shared_ptr<Ticket>& t)
    {
        if (tail) tail->next_in_stream = t;
        else head = t;
        tail = t.get();
    }
    std::shared_ptr<Ticket> pop()
    {
        std::shared_ptr<Ticket> t = std::move(head);
        head = std::move(t->next_in_stream);
        if (!head) tail = nullptr;
        return t;
    }
};

// Live tickets by id in O(1) without hashing: an id is
// (submission sequence << kSlotBits) | slot, so ids grow in submission order
// and the slot is read off the id (its ticket must carry the same id).
class TicketTable {
public:
    static constexpr int kSlotBits = 24;
    static constexpr uint64_t kSlotMask = (uint64_t(1) << kSlotBits) - 1;
    void reserve(size_t n) { slots_.reserve(n); }
    // Gives t the id of sequence number seq and a free slot; false when all
    // 2^24 slots hold live tickets.
    bool insert(const std::shared_ptr<Ticket>& t, uint64_t seq)
    {
        uint32_t slot;
        if (!free_.empty()) {
            slot = free_.back();
            free_.pop_back();
        } else {
            if (slots_.size() > kSlotMask) return false;
            slot = (uint32_t)slots_.size();
            slots_.emplace_back();
        }
        t->id = (seq << kSlotBits) | slot;
        slots_[slot] = t;
        return true;
    }
    std::shared_ptr<Ticket>* find(uint64_t id)
    {
        const uint64_t slot = id & kSlotMask;
        if (slot >= slots_.size()) return nullptr;
        std::shared_ptr<Ticket>& p = slots_[slot];
        return (p && p->id == id) ? &p : nullptr;
    }
    // Removes a ticket found by find(); returns it, so that the caller
    // decides where the last reference is dropped.
    std::shared_ptr<Ticket> take(std::shared_ptr<Ticket>* p)
    {
        std::shared_ptr<Ticket> t = std::move(*p);
        free_.push_back((uint32_t)(t->id & kSlotMask));
        return t;
    }

private:
    std::vector<std::shared_ptr<Ticket>> slots_;
    std::vector<uint32_t> free_;
};

enum { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };
enum { kUnclaimed = 0, kClaimedByBatch = 1, kClaimedByCancel = 2 };

class Server {
public:
    explicit Server(xg_ctx* c) : c_(c) {}
    ~Server() { stop(); }

    xg_status start(const xg_server_config& cfg)
    {
        cfg_ = cfg;
        if (cfg_.mem_cap_bytes == 0) cfg_.mem_cap_bytes = size_t(16) << 30;
        if (cfg_.max_batch == 0) cfg_.max_batch = 1024;
        if (cfg_.lanes == 0) cfg_.lanes = 48;
        if (cfg_.lanes > 64) return fail(XG_EINVAL, "at most 64 lanes");
        if (xg_status s = pool_.init(cfg_.mem_cap_bytes)) return s;
        const size_t nflags = (size_t)cfg_.lanes * cfg_.max_batch;
        if (cudaHostAlloc(reinterpret_cast<void**>(&h_flags_), nflags * 4, cudaHostAllocMapped) != cudaSuccess)
            return fail(XG_ENOMEM, "server: pinned flag allocation failed");
        std::memset(h_flags_, 0, nflags * 4);
        if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_flags_), h_flags_, 0) != cudaSuccess)
            return fail(XG_ECUDA, "server: cudaHostGetDevicePointer failed");
        queues_.assign(c_->n, StreamQueue());
        tickets_.reserve(size_t(1) << 16);
        lanes_.resize(cfg_.lanes);
        for (auto& l : lanes_) {
            l.launcher = std::make_unique<BatchLauncher>();
            if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess)
                return fail(XG_ECUDA, "server: stream creation failed");
            if (xg_status s = l.launcher->reserve(c_, cfg_.max_batch)) return fail(s, "server: batch launcher");
            // room for requests cut into pieces, so the first ones do not allocate
            if (xg_status s = l.launcher->reserve_jump(2048, 4096)) return fail(s, "server: jump buffers");
        }
        // the jump powers a cut request can need (pieces of 2^15..2^22 words,
        // calls up to 2^32 words), built now rather than on the first request
        for (int k = 0; k <= 32; ++k) {
            xg_status st = XG_OK;
            if (!jump_matrix(c_->device, (int)c_->param_set, k, lanes_[0].stream, &st)) return st;
        }
        // host-side fault injection for tests: the first N batch launches
        // report failure without reaching the GPU
        if (const char* f = std::getenv("XG_INJECT_LAUNCH_FAILURES")) inject_failures_ = std::atoi(f);
        // optional per-batch trace, written as CSV when the server stops
        if (const char* f = std::getenv("XG_SERVER_TRACE")) {
            trace_path_ = f;
            for (auto& l : lanes_)
                if (cudaEventCreate(&l.ev0) != cudaSuccess || cudaEventCreate(&l.ev1) != cudaSuccess)
                    return fail(XG_ECUDA, "server: trace event creation failed");
        }
        run_ = true;
        th_ = std::thread([this] { loop(); });
        return XG_OK;
    }

    void stop()
    {
        if (run_.exchange(false)) {
            cv_.notify_all();
            if (th_.joinable()) th_.join();
        }
        for (auto& l : lanes_) {
            if (l.stream) {
                cudaStreamSynchronize(l.stream);
                l.launcher.reset();
                cudaStreamDestroy(l.stream);
                l.stream = nullptr;
            }
            if (l.ev0) cudaEventDestroy(l.ev0);
            if (l.ev1) cudaEventDestroy(l.ev1);
            l.ev0 = l.ev1 = nullptr;
        }
        lanes_.clear();
        write_trace();
        if (h_flags_) cudaFreeHost(h_flags_);
        h_flags_ = nullptr;
    }

    xg_status submit(const xg_request& r, uint64_t* ticket)
    {
        if (!ticket) return fail(XG_EINVAL, "null ticket");
        if (r.stream >= c_->n) return fail(XG_EINVAL, "stream %u out of range", r.stream);
        if (r.type > XG_NORMAL_F32) return fail(XG_EINVAL, "unknown type %u", r.type);
        if (r.count == 0) return fail(XG_EINVAL, "empty request");
        if (r.count > cfg_.mem_cap_bytes / 4)
            return fail(XG_EINVAL, "request of %llu outputs exceeds the memory cap (%llu bytes): it could never be admitted",
                        (unsigned long long)r.count, (unsigned long long)cfg_.mem_cap_bytes);
        if (reinterpret_cast<uintptr_t>(r.d_out) & 3u) return fail(XG_EINVAL, "output not 4-byte aligned");
        auto t = std::make_shared<Ticket>();
        t->req = r;
        t->bytes = (size_t)r.count * 4;
        std::lock_guard<std::mutex> lk(adm_mu_);
        if (outstanding_ + t->bytes > cfg_.mem_cap_bytes) {
            ++refused_;
            return fail(XG_EAGAIN, "admission refused: %zu bytes outstanding, cap %llu", outstanding_,
                        (unsigned long long)cfg_.mem_cap_bytes);
        }
        if (r.d_out) {
            t->out = r.d_out;
        } else {
            t->out = pool_.alloc(t->bytes, &t->pool_block);
            if (!t->out) {
                ++refused_;
                return fail(XG_EAGAIN, "admission refused: no pool block of %zu bytes", t->bytes);
            }
            t->pooled = true;
        }
        t->seq = next_seq_++;
        if (!tickets_.insert(t, t->seq)) {
            if (t->pooled) pool_.release(t->pool_block);
            ++refused_;
            return fail(XG_EAGAIN, "admission refused: 2^24 tickets outstanding");
        }
        outstanding_ += t->bytes;
        t->t_submit = now_ns();
        ++submitted_;
        *ticket = t->id;
        {
            // nested (admission, then queue): per stream, queue order is ticket order
            std::lock_guard<std::mutex> ql(mu_);
            incoming_.push_back(t);
        }
        cv_.notify_one();
        return XG_OK;
    }

    // Admit reqs[0..n) in order under one lock, stopping at the first one the
    // cap or the pool refuses.  All are validated first: an invalid request
    // admits none.
    xg_status submit_many(const xg_request* reqs, uint32_t n, uint64_t* tickets, uint32_t* n_accepted)
    {
        *n_accepted = 0;
        for (uint32_t i = 0; i < n; ++i) {
            const xg_request& r = reqs[i];
            if (r.stream >= c_->n) return fail(XG_EINVAL, "request %u: stream %u out of range", i, r.stream);
            if (r.type > XG_NORMAL_F32) return fail(XG_EINVAL, "request %u: unknown type %u", i, r.type);
            if (r.count == 0) return fail(XG_EINVAL, "request %u: empty request", i);
            if (r.count > cfg_.mem_cap_bytes / 4)
                return fail(XG_EINVAL, "request %u: %llu outputs exceed the memory cap (%llu bytes)", i,
                            (unsigned long long)r.count, (unsigned long long)cfg_.mem_cap_bytes);
            if (reinterpret_cast<uintptr_t>(r.d_out) & 3u)
                return fail(XG_EINVAL, "request %u: output not 4-byte aligned", i);
        }
        std::vector<std::shared_ptr<Ticket>> made;
        made.reserve(n);
        std::lock_guard<std::mutex> lk(adm_mu_);
        const uint64_t now = now_ns();
        uint32_t k = 0;
        for (; k < n; ++k) {
            // tickets only for the requests admitted (a refused tail makes none)
            const size_t bytes = (size_t)reqs[k].count * 4;
            if (outstanding_ + bytes > cfg_.mem_cap_bytes) break;
            void* out = reqs[k].d_out;
            const bool pooled = out == nullptr;
            uint32_t block = 0;
            if (pooled) {
                out = pool_.alloc(bytes, &block);
                if (!out) break;
            }
            auto t = std::make_shared<Ticket>();
            t->req = reqs[k];
            t->bytes = bytes;
            t->out = out;
            t->pooled = pooled;
            t->pool_block = block;
            t->seq = next_seq_;
            if (!tickets_.insert(t, t->seq)) {
                if (pooled) pool_.release(block);
                break;
            }
            ++next_seq_;
            outstanding_ += t->bytes;
            t->t_submit = now;
            tickets[k] = t->id;
            made.push_back(std::move(t));
        }
        submitted_ += k;
        *n_accepted = k;
        if (k) {
            {
                std::lock_guard<std::mutex> ql(mu_);
                incoming_.insert(incoming_.end(), made.begin(), made.begin() + k);
            }
            cv_.notify_one();
        }
        if (k < n) {
            ++refused_;
            return fail(XG_EAGAIN, "admission refused at request %u: %zu bytes outstanding, cap %llu", k,
                        outstanding_, (unsigned long long)cfg_.mem_cap_bytes);
        }
        return XG_OK;
    }

    std::shared_ptr<Ticket> find(uint64_t id)
    {
        std::lock_guard<std::mutex> lk(adm_mu_);
        std::shared_ptr<Ticket>* p = tickets_.find(id);
        return p ? *p : nullptr;
    }

    bool check_flag(Ticket& t)
    {
        const int st = t.state.load(std::memory_order_acquire);
        if (st == kDone || st == kFailed || st == kCancelled) return true;
        if (t.state.load(std::memory_order_acquire) != kRunning) return false;
        volatile uint32_t* f = h_flags_ + t.slot;
        if (*f < t.expected) return false;
        int expect = kRunning;
        if (t.state.compare_exchange_strong(expect, kDone)) t.t_done.store(now_ns());
        return true;
    }

    xg_status poll(uint64_t id, int* done, void** out)
    {
        auto t = find(id);
        if (!t) return fail(XG_ENOTFOUND, "unknown ticket %llu", (unsigned long long)id);
        const bool d = check_flag(*t);
        if (t->state.load() == kFailed) return fail(XG_EDEVICE, "ticket %llu failed: its batch did not run",
                                                    (unsigned long long)id);
        if (t->state.load() == kCancelled)
            return fail(XG_ECANCELED, "ticket %llu was cancelled", (unsigned long long)id);
        if (done) *done = d ? 1 : 0;
        if (out) *out = d ? t->out : nullptr;
        return XG_OK;
    }

    xg_status wait(uint64_t id, uint32_t timeout_ms, void** out)
    {
        auto t = find(id);
        if (!t) return fail(XG_ENOTFOUND, "unknown ticket %llu", (unsigned long long)id);
        const uint64_t deadline = now_ns() + (uint64_t)timeout_ms * 1000000ull;
        while (!check_flag(*t)) {
            if (now_ns() > deadline) return fail(XG_ETIMEDOUT, "ticket %llu not done after %u ms",
                                                 (unsigned long long)id, timeout_ms);
            std::this_thread::yield();
        }
        if (t->state.load() == kFailed) return fail(XG_EDEVICE, "ticket %llu failed: its batch did not run",
                                                    (unsigned long long)id);
        if (t->state.load() == kCancelled)
            return fail(XG_ECANCELED, "ticket %llu was cancelled", (unsigned long long)id);
        if (out) *out = t->out;
        return XG_OK;
    }

    xg_status cancel(uint64_t id)
    {
        auto t = find(id);
        if (!t) return fail(XG_ENOTFOUND, "unknown ticket %llu", (unsigned long long)id);
        int expect = kUnclaimed;
        if (!t->claim.compare_exchange_strong(expect, kClaimedByCancel))
            return fail(XG_EINVAL, "ticket %llu is already launched or cancelled", (unsigned long long)id);
        // the scheduler drops it from its stream's queue when it reaches it
        t->state.store(kCancelled, std::memory_order_release);
        t->t_done.store(now_ns());
        return XG_OK;
    }

    xg_status release(uint64_t id)
    {
        std::lock_guard<std::mutex> lk(adm_mu_);
        std::shared_ptr<Ticket>* p = tickets_.find(id);
        if (!p) return fail(XG_ENOTFOUND, "unknown ticket %llu", (unsigned long long)id);
        Ticket& t = **p;
        if (t.state.load() != kDone && t.state.load() != kFailed && t.state.load() != kCancelled) {
            // the scheduler may not have seen the flag yet
            volatile uint32_t* f = h_flags_ + t.slot;
            if (!(t.state.load() == kRunning && *f >= t.expected))
                return fail(XG_EINVAL, "ticket %llu still in flight", (unsigned long long)id);
        }
        if (t.pooled) pool_.release(t.pool_block);
        outstanding_ -= t.bytes;
        tickets_.take(p);
        return XG_OK;
    }

    xg_status times(uint64_t id, uint64_t* ts, uint64_t* tl, uint64_t* td)
    {
        auto t = find(id);
        if (!t) return fail(XG_ENOTFOUND, "unknown ticket %llu", (unsigned long long)id);
        check_flag(*t);
        if (ts) *ts = t->t_submit;
        if (tl) *tl = t->t_launch;
        if (td) *td = t->t_done.load();
        return XG_OK;
    }

    // Up to max finished tickets, oldest completion first; optionally
    // released as well.
    xg_status collect(xg_completion* out, uint32_t max, uint32_t* n_out, int release)
    {
        uint32_t n = 0;
        std::vector<std::shared_ptr<Ticket>> got;
        {
            // take up to max finished tickets in one go
            std::lock_guard<std::mutex> dl(done_mu_);
            const size_t k = std::min<size_t>(max, done_q_.size());
            got.assign(std::make_move_iterator(done_q_.begin()), std::make_move_iterator(done_q_.begin() + k));
            done_q_.erase(done_q_.begin(), done_q_.begin() + k);
        }
        std::vector<std::shared_ptr<Ticket>> dropped;   // freed after the lock is released
        std::lock_guard<std::mutex> lk(adm_mu_);
        for (auto& t : got) {
            std::shared_ptr<Ticket>* p = tickets_.find(t->id);
            if (!p) continue;  // already released by its owner
            xg_completion& c = out[n++];
            c.ticket = t->id;
            c.t_submit_ns = t->t_submit;
            c.t_launch_ns = t->t_launch;
            c.t_done_ns = t->t_done.load();
            const int tst = t->state.load();
            c.status = tst == kDone ? XG_OK : tst == kCancelled ? XG_ECANCELED : XG_EDEVICE;
            c.pad = 0;
            c.d_result = t->out;
            if (release) {
                if (t->pooled) pool_.release(t->pool_block);
                outstanding_ -= t->bytes;
                dropped.push_back(tickets_.take(p));
                c.d_result = nullptr;
            }
        }
        *n_out = n;
        return XG_OK;   // lk unlocks before dropped (declared earlier) frees the tickets
    }

    void stats(xg_server_stats* s)
    {
        std::lock_guard<std::mutex> lk(adm_mu_);
        s->submitted = submitted_;
        s->completed = completed_.load();
        s->refused = refused_;
        s->outstanding_bytes = outstanding_;
        s->batches = batches_.load();
        s->items_launched = items_launched_.load();
        s->queued = queued_.load();
        s->in_flight = in_flight_.load();
        s->now_ns = now_ns();
        s->host_launch_ns = launch_ns_.load();
    }

private:
    struct Lane {
        cudaStream_t stream = nullptr;
        std::unique_ptr<BatchLauncher> launcher;
        std::vector<std::shared_ptr<Ticket>> inflight;
        bool busy = false;
        uint64_t words = 0;  // words of the batch in flight
        // tracing (XG_SERVER_TRACE): GPU start/end of the batch in flight
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        uint64_t t_launch = 0, t_host = 0;
        uint32_t n_items = 0, n_units = 0;
    };
    struct TraceRec {
        uint32_t lane, items, units;
        uint64_t words, t_launch_ns, host_ns, t_seen_done_ns;
        float gpu_ms;
    };

    // Shortest piece a new batch may cut its calls into, from the words the
    // GPU already has in flight: cutting shortens one call's critical path
    // but costs jump-ahead work (about 2.2e4 words' worth per piece), which
    // only pays while the GPU would otherwise idle.  B is about 1.5 ms of
    // work: 2^18 words for each of 32 warps per SM.  2^15 only while the GPU
    // is nearly idle (below B/32): at about a third of the GPU's rate the
    // extra jump-ahead of 2^15-word pieces tripled the p99 against 2^16.
    uint64_t min_piece_for_backlog() const
    {
        const uint64_t B = (uint64_t)c_->sm_count * 32 * (uint64_t(1) << 18);
        if (inflight_words_ < B / 32) return BatchLauncher::kMinPiece;
        if (inflight_words_ < B / 8) return uint64_t(1) << 16;
        if (inflight_words_ < B) return uint64_t(1) << 18;
        return uint64_t(1) << 21;
    }

    void loop()
    {
        std::vector<std::shared_ptr<Ticket>> fresh;
        std::vector<HostItem> items;
        std::vector<uint32_t> units;
        const bool timed = !trace_path_.empty();
        while (run_.load()) {
            bool progress = false;
            const uint64_t q0 = timed ? now_ns() : 0;
            {
                std::unique_lock<std::mutex> lk(mu_);
                if (timed) loop_ns_[0] += now_ns() - q0;   // waiting for the lock
                if (incoming_.empty() && !any_busy() && ready_.empty()) {
                    cv_.wait_for(lk, std::chrono::milliseconds(2));
                }
                fresh.assign(incoming_.begin(), incoming_.end());
                incoming_.clear();
            }
            const uint64_t q1 = timed ? now_ns() : 0;
            ++loop_iters_;
            for (auto& t : fresh) {
                StreamQueue& q = queues_[t->req.stream];
                const bool was_empty = !q.head;
                q.push(t);
                if (was_empty && !q.busy) ready_.push({t->seq, t->req.stream});
                ++queued_;
                progress = true;
            }
            fresh.clear();
            const uint64_t q2 = timed ? now_ns() : 0;
            // completions
            for (size_t li = 0; li < lanes_.size(); ++li) {
                Lane& l = lanes_[li];
                if (!l.busy) continue;
                // finished tickets leave the lane's list (swap with the last),
                // so later scans visit only the ones still running
                for (size_t k = 0; k < l.inflight.size();) {
                    if (check_flag(*l.inflight[k])) {
                        finish(l.inflight[k]);
                        l.inflight[k] = std::move(l.inflight.back());
                        l.inflight.pop_back();
                        progress = true;
                    } else {
                        ++k;
                    }
                }
                cudaError_t e = cudaEventQuery(l.launcher->done_event());
                if (e != cudaErrorNotReady) {
                    // the batch is over: every request left is resolved now,
                    // finished if its flag has become visible meanwhile,
                    // failed (not run: launch or kernel error) otherwise
                    for (auto& t : l.inflight) {
                        if (check_flag(*t)) finish(t);
                        else fail_ticket(t);
                    }
                    if (e != cudaSuccess) cudaGetLastError();
                    if (l.ev0) {
                        float ms = -1.f;
                        // ev1 follows the batch's own completion event: done at most a moment later
                        if (cudaEventSynchronize(l.ev1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, l.ev0, l.ev1) != cudaSuccess) {
                            cudaGetLastError();
                            ms = -1.f;
                        }
                        trace_.push_back(TraceRec{(uint32_t)li, l.n_items, l.n_units, l.words, l.t_launch, l.t_host,
                                                  now_ns(), ms});
                    }
                    l.busy = false;
                    l.inflight.clear();
                    l.words = 0;
                    progress = true;
                }
            }
            const uint64_t q3 = timed ? now_ns() : 0;
            // launches.  While the GPU already has about 1.5 ms of work in
            // flight, new requests wait and gather into larger batches (an
            // earlier launch would only queue behind that work).
            const uint64_t busy_words = (uint64_t)c_->sm_count * 32 * (uint64_t(1) << 18);
            for (size_t li = 0; li < lanes_.size() && !ready_.empty() && inflight_words_ < busy_words; ++li) {
                Lane& l = lanes_[li];
                if (l.busy) continue;
                items.clear();
                l.inflight.clear();
                std::memset(h_flags_ + li * cfg_.max_batch, 0, (size_t)cfg_.max_batch * 4);
                const uint64_t t_launch = now_ns();
                uint64_t batch_words = 0;
                while (!ready_.empty() && items.size() < cfg_.max_batch) {
                    const uint32_t s = ready_.top().second;
                    ready_.pop();
                    StreamQueue& q = queues_[s];
                    auto t = q.pop();
                    int expect = kUnclaimed;
                    if (!t->claim.compare_exchange_strong(expect, kClaimedByBatch)) {
                        // cancelled: never runs; the stream's next request is ready
                        --queued_;
                        if (q.head) ready_.push({q.head->seq, s});
                        std::lock_guard<std::mutex> dl(done_mu_);
                        done_q_.push_back(std::move(t));
                        continue;
                    }
                    q.busy = true;
                    t->slot = (uint32_t)(li * cfg_.max_batch + items.size());
                    t->t_launch = t_launch;
                    items.push_back(HostItem{s, t->req.type, t->req.count, t->out, d_flags_ + t->slot});
                    batch_words += t->req.count;
                    l.inflight.push_back(t);
                    --queued_;
                }
                if (items.empty()) continue;
                in_flight_ += items.size();
                const uint64_t min_piece = min_piece_for_backlog();
                inflight_words_ += batch_words;   // finish() takes each request's share back
                units.resize(items.size());
                xg_status lst = XG_ECUDA;
                if (inject_failures_ > 0) --inject_failures_;
                else {
                    const uint64_t h0 = now_ns();
                    if (l.ev0) cudaEventRecord(l.ev0, l.stream);
                    lst = l.launcher->launch(c_, items.data(), (uint32_t)items.size(), l.stream, units.data(),
                                             min_piece);
                    if (l.ev1) cudaEventRecord(l.ev1, l.stream);
                    const uint64_t h1 = now_ns();
                    launch_ns_ += h1 - h0;
                    l.t_launch = h0;
                    l.t_host = h1 - h0;
                    l.n_items = (uint32_t)items.size();
                    l.n_units = 0;
                    for (uint32_t u : units) l.n_units += u;
                }
                for (size_t j = 0; j < l.inflight.size(); ++j) {
                    l.inflight[j]->expected = lst == XG_OK ? units[j] : 1u;
                    l.inflight[j]->state.store(kRunning, std::memory_order_release);
                }
                if (lst != XG_OK) {
                    cudaGetLastError();
                    launch_error_ = true;
                    for (auto& t : l.inflight) fail_ticket(t);
                    l.inflight.clear();
                    continue;
                }
                l.busy = true;
                l.words = batch_words;
                ++batches_;
                items_launched_ += items.size();
                progress = true;
            }
            if (timed) {
                const uint64_t q4 = now_ns();
                loop_ns_[1] += q2 - q1;   // queueing new requests
                loop_ns_[2] += q3 - q2;   // completion scan
                loop_ns_[3] += q4 - q3;   // launches
            }
            if (!progress) std::this_thread::yield();
        }
    }

    void write_trace()
    {
        if (trace_path_.empty()) return;
        if (FILE* f = std::fopen(trace_path_.c_str(), "w")) {
            std::fprintf(f, "lane,items,units,words,t_launch_ns,host_ns,t_seen_done_ns,gpu_ms\n");
            std::fprintf(f, "# loop iterations %llu; ns waiting for the lock %llu, queueing %llu, "
                            "completion scan %llu, launches %llu\n",
                         (unsigned long long)loop_iters_, (unsigned long long)loop_ns_[0],
                         (unsigned long long)loop_ns_[1], (unsigned long long)loop_ns_[2],
                         (unsigned long long)loop_ns_[3]);
            for (const TraceRec& r : trace_)
                std::fprintf(f, "%u,%u,%u,%llu,%llu,%llu,%llu,%.4f\n", r.lane, r.items, r.units,
                             (unsigned long long)r.words, (unsigned long long)r.t_launch_ns,
                             (unsigned long long)r.host_ns, (unsigned long long)r.t_seen_done_ns, r.gpu_ms);
            std::fclose(f);
        }
        trace_.clear();
        trace_path_.clear();  // stop() may run again (destructor): write once
    }

    bool any_busy() const
    {
        for (auto& l : lanes_)
            if (l.busy) return true;
        return false;
    }

    void fail_ticket(const std::shared_ptr<Ticket>& t)
    {
        int expect = kRunning;
        if (t->state.compare_exchange_strong(expect, kFailed)) t->t_done.store(now_ns());
        finish(t);
    }

    void finish(const std::shared_ptr<Ticket>& t)
    {
        const uint32_t s = t->req.stream;
        inflight_words_ -= t->req.count;
        StreamQueue& q = queues_[s];
        q.busy = false;
        if (q.head) ready_.push({q.head->seq, s});
        ++completed_;
        --in_flight_;
        std::lock_guard<std::mutex> dl(done_mu_);
        done_q_.push_back(t);
    }

    xg_ctx* c_;
    xg_server_config cfg_{};
    DevicePool pool_;
    std::mutex adm_mu_;  // admission: outstanding_, pool_, tickets_, counters (taken before mu_)
    std::mutex mu_;      // incoming_ and cv_
    std::condition_variable cv_;
    TicketTable tickets_;
    std::deque<std::shared_ptr<Ticket>> incoming_;
    uint64_t next_seq_ = 1;
    size_t outstanding_ = 0;
    uint64_t submitted_ = 0, refused_ = 0;
    std::atomic<uint64_t> completed_{0}, batches_{0}, items_launched_{0}, queued_{0}, in_flight_{0};
    std::atomic<uint64_t> launch_ns_{0};
    std::atomic<bool> launch_error_{false};
    int inject_failures_ = 0;
    std::mutex done_mu_;
    std::deque<std::shared_ptr<Ticket>> done_q_;  // finished, not yet collected
    uint64_t inflight_words_ = 0;                 // scheduler thread only
    std::string trace_path_;
    uint64_t loop_iters_ = 0, loop_ns_[4] = {0, 0, 0, 0};  // scheduler thread only
    std::vector<TraceRec> trace_;                 // scheduler thread until stop
    // scheduler thread only
    std::vector<StreamQueue> queues_;  // one per stream of the context
    std::priority_queue<std::pair<uint64_t, uint32_t>, std::vector<std::pair<uint64_t, uint32_t>>,
                        std::greater<std::pair<uint64_t, uint32_t>>>
        ready_;
    std::vector<Lane> lanes_;
    uint32_t* h_flags_ = nullptr;
    uint32_t* d_flags_ = nullptr;
    std::thread th_;
    std::atomic<bool> run_{false};

    friend void ::xg_ctx::shutdown_server();
};

}  // namespace xg

void xg_ctx::shutdown_server()
{
    if (server) {
        server->stop();
        delete server;
        server = nullptr;
    }
}

using xg::fail;

extern "C" {

xg_status xg_server_start(xg_ctx* ctx, const xg_server_config* cfg)
{
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (ctx->server) return fail(XG_EINVAL, "server already running");
    xg_server_config c{};
    if (cfg) c = *cfg;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStreamSynchronize(ctx->stream);
    auto* s = new (std::nothrow) xg::Server(ctx);
    if (!s) return fail(XG_ENOMEM, "host allocation failed");
    if (xg_status st = s->start(c)) {
        delete s;
        return st;
    }
    ctx->server = s;
    return XG_OK;
}

xg_status xg_server_stop(xg_ctx* ctx)
{
    if (!ctx) return fail(XG_EINVAL, "null context");
    ctx->shutdown_server();
    return XG_OK;
}

xg_status xg_submit(xg_ctx* ctx, const xg_request* req, uint64_t* ticket)
{
    if (!ctx || !req) return fail(XG_EINVAL, "null argument");
    if (!ctx->server) return fail(XG_EINVAL, "server not running (xg_server_start)");
    return ctx->server->submit(*req, ticket);
}

xg_status xg_submit_many(xg_ctx* ctx, const xg_request* reqs, uint32_t n, uint64_t* tickets, uint32_t* n_accepted)
{
    if (!ctx || !n_accepted || (n && (!reqs || !tickets))) return fail(XG_EINVAL, "null argument");
    *n_accepted = 0;
    if (!ctx->server) return fail(XG_EINVAL, "server not running (xg_server_start)");
    if (n == 0) return XG_OK;
    return ctx->server->submit_many(reqs, n, tickets, n_accepted);
}

xg_status xg_poll(xg_ctx* ctx, uint64_t ticket, int* done, void** d_result)
{
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (!ctx->server) return fail(XG_EINVAL, "server not running");
    return ctx->server->poll(ticket, done, d_result);
}

xg_status xg_wait(xg_ctx* ctx, uint64_t ticket, uint32_t timeout_ms, void** d_result)
{
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (!ctx->server) return fail(XG_EINVAL, "server not running");
    return ctx->server->wait(ticket, timeout_ms, d_result);
}

xg_status xg_cancel(xg_ctx* ctx, uint64_t ticket)
{
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (!ctx->server) return fail(XG_EINVAL, "server not running");
    return ctx->server->cancel(ticket);
}

xg_status xg_release(xg_ctx* ctx, uint64_t ticket)
{
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (!ctx->server) return fail(XG_EINVAL, "server not running");
    return ctx->server->release(ticket);
}

xg_status xg_ticket_times(xg_ctx* ctx, uint64_t ticket, uint64_t* t_submit_ns, uint64_t* t_launch_ns,
                          uint64_t* t_done_ns)
{
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (!ctx->server) return fail(XG_EINVAL, "server not running");
    return ctx->server->times(ticket, t_submit_ns, t_launch_ns, t_done_ns);
}

xg_status xg_collect(xg_ctx* ctx, xg_completion* out, uint32_t max, uint32_t* n_out, int release)
{
    if (!ctx || !n_out || (max && !out)) return fail(XG_EINVAL, "null argument");
    if (!ctx->server) return fail(XG_EINVAL, "server not running");
    return ctx->server->collect(out, max, n_out, release);
}

xg_status xg_server_stats_get(xg_ctx* ctx, xg_server_stats* out)
{
    if (!ctx || !out) return fail(XG_EINVAL, "null argument");
    if (!ctx->server) return fail(XG_EINVAL, "server not running");
    ctx->server->stats(out);
    return XG_OK;
}

}  // extern "C"
