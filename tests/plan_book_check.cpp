// Randomised check of the plan table's host bookkeeping (paper_2008_03518_gb300/csrc/
// plan_book.h) against ordered containers with the same meaning: a std::set of free slots
// (the lowest is taken first), a std::map of plans by id, and an expiry that walks every
// plan. Usage: plan_book_check <seed> <slots> <window> <rounds>. Prints "ok" and exits 0
// when every step agrees; otherwise prints the first disagreement and exits 1.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <set>

#include "plan_book.h"

using fmdp::Book;
using fmdp::PlanMeta;

namespace {

struct Reference {
    std::set<int32_t> free_slots;
    std::map<uint64_t, PlanMeta> plans;
    int64_t expire(int64_t t_now) {
        int64_t n = 0;
        for (auto it = plans.begin(); it != plans.end();) {
            if (it->second.t0 + it->second.n - 1 < t_now) {
                free_slots.insert(it->second.slot);
                it = plans.erase(it);
                ++n;
            } else {
                ++it;
            }
        }
        return n;
    }
};

int fail(const char* what, long long a, long long b) {
    std::printf("mismatch: %s (%lld vs %lld)\n", what, a, b);
    return 1;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc != 5) {
        std::printf("usage: plan_book_check <seed> <slots> <window> <rounds>\n");
        return 2;
    }
    const unsigned long long seed = std::strtoull(argv[1], nullptr, 10);
    const int32_t S = (int32_t)std::atoi(argv[2]);
    const int32_t T = (int32_t)std::atoi(argv[3]);
    const int rounds = std::atoi(argv[4]);
    std::mt19937_64 rng(seed);
    Book bk;
    bk.reset(S, T);
    Reference ref;
    for (int32_t s = 0; s < S; ++s) ref.free_slots.insert(s);

    for (int round = 0; round < rounds; ++round) {
        // admissions: the lowest free slot each time, plans that stay inside the window
        const int adds = (int)(rng() % 64);
        for (int k = 0; k < adds && !ref.free_slots.empty(); ++k) {
            const int32_t s = bk.free_slots.lowest();
            if (s != *ref.free_slots.begin()) return fail("lowest free slot", s, *ref.free_slots.begin());
            bk.free_slots.erase(s);
            ref.free_slots.erase(ref.free_slots.begin());
            const int64_t t0 = bk.t_base + (int64_t)(rng() % (uint64_t)(T / 2));
            const int32_t n = 1 + (int32_t)(rng() % (uint64_t)(T / 2));
            const PlanMeta pm{s, t0, n};
            const uint64_t id = bk.next_id++;
            bk.add(id, pm);
            ref.plans[id] = pm;
            if (s + 1 > bk.S_hw) bk.S_hw = s + 1;
        }
        // removals by id (a rolled-back admission), the slot freed by the caller
        const int dels = (int)(rng() % 16);
        for (int k = 0; k < dels && !ref.plans.empty(); ++k) {
            auto it = ref.plans.begin();
            std::advance(it, (long)(rng() % ref.plans.size()));
            if (!bk.erase(it->first)) return fail("erase of a live id", (long long)it->first, 0);
            bk.free_slots.insert(it->second.slot);
            ref.free_slots.insert(it->second.slot);
            ref.plans.erase(it);
        }
        if (bk.erase(bk.next_id + 7)) return fail("erase of an unknown id", 1, 0);
        // expiry: usually a few steps, sometimes past the whole window
        const int64_t step = (rng() % 16 == 0) ? (int64_t)T + (int64_t)(rng() % 8) : (int64_t)(rng() % 24);
        const int64_t t_now = bk.t_base + step;
        const int64_t got = bk.expire(t_now), want = ref.expire(t_now);
        if (got != want) return fail("plans expired", got, want);
        bk.t_base = std::max(bk.t_base, t_now);

        if (bk.size() != ref.plans.size()) return fail("live plans", (long long)bk.size(), (long long)ref.plans.size());
        if (bk.free_slots.size() != ref.free_slots.size())
            return fail("free slots", (long long)bk.free_slots.size(), (long long)ref.free_slots.size());
        // every plan, in ascending id order, with its record
        auto rit = ref.plans.begin();
        long long visited = 0;
        bool order_ok = true;
        bk.for_each([&](uint64_t id, const PlanMeta& p) {
            if (rit == ref.plans.end() || rit->first != id || rit->second.slot != p.slot || rit->second.t0 != p.t0 ||
                rit->second.n != p.n)
                order_ok = false;
            if (rit != ref.plans.end()) ++rit;
            ++visited;
        });
        if (!order_ok || visited != (long long)ref.plans.size()) return fail("plans in id order", visited, 0);
        for (const auto& kv : ref.plans) {
            const PlanMeta* p = bk.find(kv.first);
            if (!p || p->slot != kv.second.slot) return fail("find", (long long)kv.first, 0);
        }
        // the free slots in order, from next()
        int32_t s = -1;
        for (int32_t want_s : ref.free_slots) {
            s = bk.free_slots.next(s + 1);
            if (s != want_s) return fail("next free slot", s, want_s);
        }
        if (bk.free_slots.next(s + 1) != -1) return fail("no free slot past the last", bk.free_slots.next(s + 1), -1);
        int32_t hw = 0;
        for (const auto& kv : ref.plans) hw = std::max(hw, kv.second.slot + 1);
        if (bk.slot_bound() != hw) return fail("slot bound", bk.slot_bound(), hw);
        // a copy (snapshot / restore) holds the same state
        if (round % 97 == 0) {
            const Book cp = bk;
            if (cp.size() != bk.size() || cp.free_slots.lowest() != bk.free_slots.lowest())
                return fail("copy", (long long)cp.size(), (long long)bk.size());
        }
    }
    std::printf("ok\n");
    return 0;
}
