// Host-logic check of the batch planner (no GPU): plans seeded random batches
// with the library's xg::plan_batch and verifies its invariants.  Prints
// "ok <batches> <units>" or the first violation and exits non-zero.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>

#include "xg_batch.h"

using xg::BatchItem;
using xg::BatchPlan;
using xg::HostItem;

static int fail_at(const char* what, int batch, long detail)
{
    std::printf("FAIL batch %d: %s (%ld)\n", batch, what, detail);
    return 1;
}

static uint64_t words_of(uint32_t kind, uint64_t count) { return kind == 2 ? count + (count & 1u) : count; }
static uint64_t cost_of(uint32_t kind, uint64_t w) { return w * (kind == 2 ? 18u : kind == 1 ? 9u : 8u); }

int main()
{
    std::mt19937_64 rng(486);
    BatchPlan plan;
    long total_units = 0;
    const int kBatches = 400;
    for (int b = 0; b < kBatches; ++b) {
        const uint32_t n_streams = 1 + (uint32_t)(rng() % 64);
        const uint32_t n = 1 + (uint32_t)(rng() % 200);
        const uint64_t piece = (rng() % 3 == 0) ? 0 : (uint64_t(1) << (6 + rng() % 8));  // 0 or 2^6..2^13
        std::vector<HostItem> items(n);
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t kind = (uint32_t)(rng() % 3);
            const uint64_t count = (rng() % 5 == 0) ? 0 : 1 + rng() % (uint64_t(1) << (rng() % 15));
            // most outputs 16-byte aligned, some only 4-byte aligned
            const uintptr_t off = (rng() % 4 == 0) ? 4u * (1 + rng() % 3) : 0u;
            items[i] = HostItem{(uint32_t)(rng() % n_streams), kind, count,
                                reinterpret_cast<void*>((uintptr_t)(0x100000000ull * (i + 1)) + off), nullptr};
        }
        uint8_t shapes[3];
        for (auto& sh : shapes) sh = (uint8_t)(rng() % xg::kNumShapes);
        const uint64_t gmax = (b % 3 == 0) ? ~uint64_t(0) : (uint64_t(1) << (rng() % 14));
        xg::plan_batch(items.data(), n, piece, n_streams, plan, (b % 5 == 0) ? nullptr : shapes, gmax);
        // tasks: every head exactly once among the members; groups hold
        // single-unit chains of one grouped type with 16-byte aligned output
        {
            std::vector<int> head_seen(plan.units.size(), 0);
            for (uint32_t h : plan.heads) head_seen[h] = 1;
            if (plan.members.size() > plan.heads.size() + xg::kMemberSlack) return fail_at("member slack", b, 0);
            size_t listed = 0;
            for (size_t t = 0; t < plan.tasks.size(); ++t) {
                const uint32_t sh = plan.tasks[t] >> 28, first = plan.tasks[t] & xg::kTaskFirstMask;
                if (sh >= (uint32_t)xg::kNumShapes) return fail_at("task shape", b, (long)t);
                const uint32_t G = xg::shape_group(sh);
                if (first + G > plan.members.size()) return fail_at("task members range", b, (long)t);
                if (plan.members[first] == xg::kNoItem) return fail_at("empty task", b, (long)t);
                const uint32_t kind = plan.units[plan.members[first]].kind;
                bool filler = false;
                for (uint32_t g = 0; g < G; ++g) {
                    const uint32_t u = plan.members[first + g];
                    if (u == xg::kNoItem) { filler = true; continue; }
                    if (filler) return fail_at("member after filler", b, (long)t);
                    if (u >= plan.units.size() || head_seen[u] != 1) return fail_at("member not an unlisted head", b, (long)t);
                    head_seen[u] = 2;
                    ++listed;
                    if (sh != xg::kShapeChain) {
                        const BatchItem& it = plan.units[u];
                        if (it.kind != kind || kind > 1) return fail_at("group type", b, (long)t);
                        if (it.next != xg::kNoItem) return fail_at("grouped chain of several units", b, (long)t);
                        if (reinterpret_cast<uintptr_t>(it.out) & 15u) return fail_at("grouped unaligned output", b, (long)t);
                        if (words_of(it.kind, it.count) > gmax) return fail_at("grouped long unit", b, (long)t);
                        if (b % 5 == 0 || shapes[kind] != sh) return fail_at("group shape not the type's", b, (long)t);
                    }
                }
            }
            if (listed != plan.heads.size()) return fail_at("heads listed", b, (long)listed);
        }
        const uint64_t L = plan.pieces.empty() ? 0 : (uint64_t(1) << plan.split_log2);
        if (!plan.pieces.empty() && L != piece) return fail_at("piece length", b, (long)L);
        std::map<uint32_t, int> per_stream;
        for (auto& it : items) ++per_stream[it.stream];
        // walk the chains from the heads: every unit exactly once
        std::vector<int> seen(plan.units.size(), 0);
        if (plan.chain_words.size() != plan.heads.size()) return fail_at("chain cost count", b, 0);
        for (size_t h = 0; h < plan.heads.size(); ++h) {
            if (h && plan.chain_words[h] > plan.chain_words[h - 1]) {
                // ordering is by cost rounded to 7 significant bits: allow less than 1/64 inversion
                if (plan.chain_words[h] - plan.chain_words[h - 1] > plan.chain_words[h - 1] / 64 + 1)
                    return fail_at("heads not costliest first", b, (long)h);
            }
            uint64_t cost = 0;
            uint32_t stream = plan.units[plan.heads[h]].stream;
            for (uint32_t u = plan.heads[h]; u != xg::kNoItem; u = plan.units[u].next) {
                if (u >= plan.units.size()) return fail_at("unit index", b, (long)u);
                if (seen[u]++) return fail_at("unit reached twice", b, (long)u);
                if (plan.units[u].stream != stream) return fail_at("chain mixes streams", b, (long)u);
                cost += cost_of(plan.units[u].kind, words_of(plan.units[u].kind, plan.units[u].count));
            }
            if (cost != plan.chain_words[h]) return fail_at("chain cost", b, (long)h);
        }
        for (size_t u = 0; u < seen.size(); ++u)
            if (!seen[u]) return fail_at("unit not reachable", b, (long)u);
        // per item: its units cover it exactly, in order
        size_t next_unit = 0;
        for (uint32_t i = 0; i < n; ++i) {
            const HostItem& it = items[i];
            const uint64_t w = words_of(it.kind, it.count);
            const bool cut = piece && per_stream[it.stream] == 1 && w >= 2 * piece;
            const uint32_t expect_units = cut ? (uint32_t)((w + piece - 1) / piece) : 1u;
            if (plan.units_per_item[i] != expect_units) return fail_at("units per item", b, (long)i);
            uint64_t covered = 0;
            for (uint32_t k = 0; k < expect_units; ++k) {
                const BatchItem& u = plan.units[next_unit++];
                if (u.stream != it.stream || u.kind != it.kind) return fail_at("unit identity", b, (long)i);
                if (cut) {
                    const uint32_t pi = u.piece - 1;
                    if (u.piece == 0 || plan.piece_index[pi] != k || plan.piece_skip[pi] != k * piece ||
                        plan.piece_stream[pi] != it.stream)
                        return fail_at("piece record", b, (long)i);
                    if (plan.pieces[pi].item_words != w || plan.pieces[pi].last != (k + 1 == expect_units ? 1u : 0u))
                        return fail_at("piece words or last flag", b, (long)i);
                    if (reinterpret_cast<uintptr_t>(u.out) != reinterpret_cast<uintptr_t>(it.out) + 4 * k * piece)
                        return fail_at("piece output offset", b, (long)i);
                    if (u.next != xg::kNoItem) return fail_at("piece chained", b, (long)i);
                } else {
                    if (u.piece != 0 || u.count != it.count || u.out != it.out) return fail_at("whole unit", b, (long)i);
                }
                covered += u.count;
            }
            if (covered != it.count) return fail_at("coverage", b, (long)i);
        }
        if (next_unit != plan.units.size()) return fail_at("extra units", b, (long)next_unit);
        // calls on one stream run in submission order (chain order = item order)
        std::map<uint32_t, uint32_t> last_unit;
        for (size_t u = 0; u < plan.units.size(); ++u) {
            if (plan.units[u].piece) continue;
            auto f = last_unit.find(plan.units[u].stream);
            if (f != last_unit.end() && plan.units[f->second].next != u) return fail_at("chain order", b, (long)u);
            last_unit[plan.units[u].stream] = (uint32_t)u;
        }
        total_units += (long)plan.units.size();
    }
    std::printf("ok %d %ld\n", kBatches, total_units);
    return 0;
}
