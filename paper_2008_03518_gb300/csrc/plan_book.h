// Host bookkeeping of the plan table: which slot holds which plan, the free slots, and the
// plans by their last step (for expiry). Plain C++ with no CUDA types, so that its logic can
// be compiled and checked on a host without a GPU.
#pragma once

#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

namespace fmdp {

struct PlanMeta {
    int32_t slot;
    int64_t t0;
    int32_t n;
};

// Free plan slots, lowest first: one bit per slot and one summary bit per 64-slot word, so
// that taking, freeing and finding the next free slot cost a few word operations.
struct SlotPool {
    std::vector<uint64_t> bits, sum;  // bit set: slot free / word has a free slot
    int32_t cap = 0;
    size_t n = 0;
    void reset(int32_t S) {
        cap = S;
        bits.assign(((size_t)S + 63) / 64, 0);
        sum.assign((bits.size() + 63) / 64, 0);
        n = 0;
        for (int32_t s = 0; s < S; ++s) insert(s);
    }
    size_t size() const { return n; }
    bool empty() const { return n == 0; }
    void insert(int32_t s) {  // frees s (nothing if it is free)
        uint64_t& w = bits[(size_t)s >> 6];
        const uint64_t b = 1ull << (s & 63);
        if (w & b) return;
        if (!w) sum[(size_t)s >> 12] |= 1ull << ((s >> 6) & 63);
        w |= b;
        ++n;
    }
    void erase(int32_t s) {  // takes s (nothing if it is taken)
        uint64_t& w = bits[(size_t)s >> 6];
        const uint64_t b = 1ull << (s & 63);
        if (!(w & b)) return;
        w &= ~b;
        if (!w) sum[(size_t)s >> 12] &= ~(1ull << ((s >> 6) & 63));
        --n;
    }
    int32_t next(int32_t from) const {  // lowest free slot >= from, -1 if none
        if (from < 0) from = 0;
        if (from >= cap) return -1;
        const size_t wi = (size_t)from >> 6;
        const uint64_t w = bits[wi] & (~0ull << (from & 63));
        if (w) return (int32_t)(wi * 64 + __builtin_ctzll(w));
        const size_t w1 = wi + 1;
        for (size_t si = w1 >> 6; si < sum.size(); ++si) {
            uint64_t m = sum[si];
            if (si == (w1 >> 6)) m &= ~0ull << (w1 & 63);
            if (m) {
                const size_t w2 = si * 64 + __builtin_ctzll(m);
                return (int32_t)(w2 * 64 + __builtin_ctzll(bits[w2]));
            }
        }
        return -1;
    }
    int32_t lowest() const { return next(0); }
};

// Host bookkeeping of the table (copied by snapshot / restore): each slot's plan, the ids
// in the order they were given (ids only grow), and the plans by their last step modulo the
// window, so that an expiry visits only the steps it passes and finds a plan by its slot.
// An entry whose slot has since been freed or given to another plan is passed over and
// dropped (the id list is compacted when such entries outnumber the plans).
struct Book {
    SlotPool free_slots;
    std::vector<uint64_t> id_at;    // [slot] id of the slot's plan, 0 if none
    std::vector<PlanMeta> meta_at;  // [slot]
    std::vector<std::pair<uint64_t, int32_t>> by_id;                 // (id, slot), ascending ids
    std::vector<std::vector<std::pair<int32_t, uint64_t>>> by_end;  // [last step mod T] (slot, id)
    size_t live = 0;
    uint64_t next_id = 1;
    int64_t t_base = 0;
    int32_t S_hw = 0;
    void reset(int32_t S_max, int32_t T_win) {
        free_slots.reset(S_max);
        id_at.assign((size_t)S_max, 0);
        meta_at.assign((size_t)S_max, PlanMeta{});
        by_id.clear();
        by_end.assign((size_t)T_win, {});
        live = 0;
        next_id = 1;
        S_hw = 0;
    }
    size_t size() const { return live; }
    bool empty() const { return live == 0; }
    size_t end_bucket(int64_t t) const {
        const int64_t T = (int64_t)by_end.size();
        return (size_t)(((t % T) + T) % T);
    }
    void add(uint64_t id, const PlanMeta& pm) {  // id above every id added before; pm.slot free
        if (by_id.size() > 2 * live + 4096) {  // drop the entries of removed plans
            size_t k = 0;
            for (const auto& e : by_id)
                if (id_at[e.second] == e.first) by_id[k++] = e;
            by_id.resize(k);
        }
        id_at[pm.slot] = id;
        meta_at[pm.slot] = pm;
        by_id.emplace_back(id, pm.slot);
        by_end[end_bucket(pm.t0 + pm.n - 1)].emplace_back(pm.slot, id);
        ++live;
    }
    const PlanMeta* find(uint64_t id) const {
        const auto it = std::lower_bound(by_id.begin(), by_id.end(), std::make_pair(id, INT32_MIN));
        if (it == by_id.end() || it->first != id || id_at[it->second] != id) return nullptr;
        return &meta_at[it->second];
    }
    bool erase(uint64_t id) {  // removes the plan (its slot is freed by the caller)
        const PlanMeta* p = find(id);
        if (!p) return false;
        id_at[p->slot] = 0;
        --live;
        return true;
    }
    template <class F>
    void for_each(F f) const {  // f(id, plan) in ascending id order
        for (const auto& e : by_id)
            if (id_at[e.second] == e.first) f(e.first, meta_at[e.second]);
    }
    int32_t slot_bound() const {  // one past the highest slot that holds a plan
        for (int32_t s = (int32_t)id_at.size(); s > 0; --s)
            if (id_at[s - 1]) return s;
        return 0;
    }
    int64_t expire(int64_t t_now) {  // removes and frees the plans whose last step is < t_now
        if (by_end.empty() || t_now <= t_base) return 0;
        int64_t n = 0;
        const int64_t steps = std::min<int64_t>(t_now - t_base, (int64_t)by_end.size());
        for (int64_t t = t_base; t < t_base + steps; ++t) {
            auto& b = by_end[end_bucket(t)];
            size_t keep = 0;
            for (const auto& e : b) {
                if (id_at[e.first] != e.second) continue;  // removed since
                const PlanMeta& p = meta_at[e.first];
                if (p.t0 + p.n - 1 < t_now) {
                    id_at[e.first] = 0;
                    free_slots.insert(e.first);
                    --live;
                    ++n;
                } else {
                    b[keep++] = e;
                }
            }
            b.resize(keep);
        }
        return n;
    }
};

}  // namespace fmdp
