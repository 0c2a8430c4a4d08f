// pack.cpp -- the device image of a volume.
//
// The canonical buffer follows the paper's layout (Sec. 3.3).  The device
// image holds the same structures -- Raw and DF cell arrays, SVO root entries
// and child lists, SVDAG nodes -- in the same (canonical) order, relocated
// with every pointer rewritten to the new offsets, and changed in two ways:
//   - aligned: every DF cell array, SVO root entry and SVO child list starts
//     at an even word, so that a DF cell {terminating integer, distance} and
//     an SVO node entry {pointer, masks} are each read with one 8-byte load
//     (one zero word of padding where needed);
//   - packed (a format with an SVDAG level whose image stays below 2^24
//     words): a pointer to an SVDAG node carries the node's valid mask in
//     bits 24..31, which saves the dependent read of the node's masks word on
//     every descent, and an SVDAG slot of a leaf child holds the leaf's
//     terminating integer itself, so the leaf words are not stored at all.
// The image has an even number of words, so a kernel may read any cell as
// part of the 8-byte pair that starts at the even word at or below it.
// The structures read at the top node levels come first, level by level
// (canonical order within a level, and for everything below), so that the
// top k node levels of any format -- Raw, DF, SVO or SVDAG -- are one prefix
// of the image, which a kernel can stage in shared memory (stage_end).
// vx_canonical keeps returning the paper's layout; canonical_device uploads
// it unchanged (then the kernels read it with 4-byte loads).
#include <string.h>

#include <algorithm>
#include <vector>

#include "vx_internal.hpp"

namespace vx {
namespace {

enum : uint8_t { I_CELLS, I_DF, I_SVO_ROOT, I_SVO_LIST, I_DAG, I_DAG_LEAF };

struct Item {
    uint32_t old;  // canonical offset of the structure's first word
    uint32_t len;  // words
    uint8_t kind, level, depth, align;  // depth: SVO list entries' / SVDAG node's octree depth
};

class Relocator {
  public:
    Relocator(const Spec& sp, const std::vector<uint32_t>& in) : sp_(sp), in_(in), seen_(in.size(), 0) {
        nlev_ = (int)sp.lv.size();
        int j = 0;
        for (int k = 0; k < nlev_; k++) {
            j0_[k] = j;
            j += sp.lv[k].kind == K_SVO || sp.lv[k].kind == K_DAG ? sp.lv[k].e[0] : 1;
        }
    }

    // stage_end[k] (k = 0..kStageLevels): the image's words before the
    // first structure read at node level k or deeper
    uint32_t stage_end[kStageLevels + 1] = {};

    // Builds the image; false if the buffer is not a well-formed volume of
    // the spec or an offset would not fit 32 bits (the caller then uploads
    // the canonical words).
    bool run(std::vector<uint32_t>& out, bool& packed) {
        packed = false;
        if (in_.empty()) return false;
        if (in_[0] == 0) {
            out.assign(1, 0u);
            return true;
        }
        level(0, in_[0]);
        if (!ok_) return false;
        std::sort(items_.begin(), items_.end(), [](const Item& a, const Item& b) { return a.old < b.old; });
        // placement: the structures read at node levels 0 .. kStageLevels - 1
        // first, level by level, then the rest; canonical order within each
        order_.resize(items_.size());
        for (size_t i = 0; i < items_.size(); i++) order_[i] = (uint32_t)i;
        std::stable_sort(order_.begin(), order_.end(),
                         [&](uint32_t a, uint32_t b) { return stage(items_[a]) < stage(items_[b]); });
        bool any_dag = false;
        for (const Level& L : sp_.lv) any_dag |= L.kind == K_DAG;
        uint64_t size = assign(any_dag);
        packed = any_dag && size < (1ull << 24);
        if (any_dag && !packed) size = assign(false);
        size += size & 1;  // an even number of words: every aligned 8-byte pair lies inside
        if (size > 0xFFFFFFFFull) return false;
        out.assign((size_t)size, 0u);
        out[0] = ptr_to(0, in_[0], packed);
        for (const Item& it : items_) write(it, out, packed);
        return ok_;
    }

  private:
    bool check(uint64_t p, uint64_t n) {
        if (p == 0 || p + n > in_.size()) ok_ = false;
        return ok_;
    }
    bool first_visit(uint32_t p) {
        if (seen_[p]) return false;
        seen_[p] = 1;
        return true;
    }
    void add(uint32_t p, uint64_t n, uint8_t kind, int k, int depth, int align) {
        items_.push_back(Item{p, (uint32_t)n, kind, (uint8_t)k, (uint8_t)depth, (uint8_t)align});
    }

    // ---- pass 1: every structure reachable from the root, once ----
    void level(int k, uint32_t p) {
        if (!ok_ || !check(p, 1) || !first_visit(p)) return;
        const Level& L = sp_.lv[k];
        const bool last = k == nlev_ - 1;
        if (L.kind == K_RAW || L.kind == K_DF) {
            const uint64_t cells = 1ull << (L.e[0] + L.e[1] + L.e[2]);
            const uint64_t wpc = L.kind == K_DF ? 2 : 1;  // DF: {terminating integer, distance}
            if (!check(p, wpc * cells)) return;
            add(p, wpc * cells, L.kind == K_DF ? I_DF : I_CELLS, k, 0, L.kind == K_DF ? 2 : 1);
            if (last) return;
            for (uint64_t i = 0; i < cells && ok_; i++) {
                const uint32_t w = in_[p + wpc * i];
                if (w) level(k + 1, w);
            }
        } else if (L.kind == K_SVO) {
            if (!check(p, 2)) return;
            add(p, 2, I_SVO_ROOT, k, 0, 2);
            svo_list(k, in_[p], in_[p + 1] & 0xFFu, 1);
        } else {
            dag(k, p, 0);
        }
    }
    // child list at `first` of a node with valid mask `valid`: its entries sit
    // at octree depth dd (leaves when dd == L)
    void svo_list(int k, uint32_t first, uint32_t valid, int dd) {
        const uint32_t cnt = (uint32_t)__builtin_popcount(valid);
        if (!ok_ || cnt == 0 || !check(first, 2ull * cnt) || !first_visit(first)) return;
        const int L = sp_.lv[k].e[0];
        const bool last = k == nlev_ - 1;
        add(first, 2ull * cnt, I_SVO_LIST, k, dd, 2);
        for (uint32_t r = 0; r < cnt && ok_; r++) {
            const uint32_t c = first + 2 * r;
            if (dd == L) {
                if (!last) level(k + 1, in_[c]);
            } else {
                svo_list(k, in_[c], in_[c + 1] & 0xFFu, dd + 1);
            }
        }
    }
    void dag(int k, uint32_t p, int d) {
        if (!ok_ || !check(p, 1)) return;
        if (d > 0 && !first_visit(p)) return;  // roots were marked by level()
        const int L = sp_.lv[k].e[0];
        const bool last = k == nlev_ - 1;
        const uint32_t cnt = (uint32_t)__builtin_popcount(in_[p] & 0xFFu);
        if (!check(p, 1ull + cnt)) return;
        add(p, 1ull + cnt, I_DAG, k, d, 1);
        for (uint32_t r = 0; r < cnt && ok_; r++) {
            const uint32_t c = in_[p + 1 + r];
            if (!check(c, 1)) return;
            if (d + 1 == L) {
                if (!first_visit(c)) continue;
                add(c, 1, I_DAG_LEAF, k, L, 1);
                if (!last) level(k + 1, in_[c]);
            } else {
                dag(k, c, d + 1);
            }
        }
    }

    // node level whose walk reads the structure, capped at kStageLevels
    int stage(const Item& it) const {
        const int j0 = j0_[it.level];
        int j = j0;
        if (it.kind == I_SVO_LIST) j = j0 + it.depth - 1;          // read by its parent's descent
        else if (it.kind == I_DAG) j = j0 + it.depth;               // its slots, at its own level
        else if (it.kind == I_DAG_LEAF) j = j0 + it.depth - 1;      // read from a slot one level up
        return j < kStageLevels ? j : kStageLevels;
    }

    // ---- new offsets in placement order; returns the image size ----
    uint64_t assign(bool packed) {
        newoff_.assign(items_.size(), 0u);
        uint64_t cur = 1;  // word 0: root pointer
        int next_stage = 0;
        for (uint32_t i : order_) {
            const Item& it = items_[i];
            while (next_stage <= stage(it) && next_stage <= kStageLevels)
                stage_end[next_stage++] = (uint32_t)std::min<uint64_t>(cur, 0xFFFFFFFFull);
            if (packed && it.kind == I_DAG_LEAF) continue;  // inlined into the slots
            if (it.align == 2 && (cur & 1)) cur++;
            newoff_[i] = (uint32_t)std::min<uint64_t>(cur, 0xFFFFFFFFull);
            cur += it.len;
        }
        while (next_stage <= kStageLevels) stage_end[next_stage++] = (uint32_t)std::min<uint64_t>(cur, 0xFFFFFFFFull);
        return cur;
    }
    uint32_t where(uint32_t old) {
        auto pos = std::lower_bound(items_.begin(), items_.end(), old,
                                    [](const Item& a, uint32_t v) { return a.old < v; });
        if (pos == items_.end() || pos->old != old) {
            ok_ = false;
            return 0;
        }
        return newoff_[pos - items_.begin()];
    }
    // the word a parent stores for the root of level k's sub-volume at canonical p
    uint32_t ptr_to(int k, uint32_t p, bool packed) {
        const uint32_t n = where(p);
        if (packed && sp_.lv[k].kind == K_DAG) return ((in_[p] & 0xFFu) << 24) | n;
        return n;
    }

    // ---- pass 2: copy each structure, pointers rewritten ----
    void write(const Item& it, std::vector<uint32_t>& out, bool packed) {
        if (packed && it.kind == I_DAG_LEAF) return;
        const uint32_t* src = in_.data() + it.old;
        uint32_t* dst = out.data() + where(it.old);
        const int k = it.level;
        const bool last = k == nlev_ - 1;
        const int L = sp_.lv[k].e[0];
        switch (it.kind) {
            case I_CELLS:
                for (uint32_t i = 0; i < it.len; i++) dst[i] = (last || !src[i]) ? src[i] : ptr_to(k + 1, src[i], packed);
                break;
            case I_DF:
                for (uint32_t i = 0; i < it.len; i += 2) {
                    dst[i] = (last || !src[i]) ? src[i] : ptr_to(k + 1, src[i], packed);
                    dst[i + 1] = src[i + 1];
                }
                break;
            case I_SVO_ROOT:
                dst[0] = where(src[0]);
                dst[1] = src[1];
                break;
            case I_SVO_LIST:
                for (uint32_t i = 0; i < it.len; i += 2) {
                    if (it.depth == L) dst[i] = last ? src[i] : ptr_to(k + 1, src[i], packed);
                    else dst[i] = where(src[i]);
                    dst[i + 1] = src[i + 1];
                }
                break;
            case I_DAG:
                dst[0] = src[0];
                for (uint32_t r = 1; r < it.len; r++) {
                    const uint32_t c = src[r];
                    if (it.depth + 1 == L) {
                        if (packed) dst[r] = last ? in_[c] : ptr_to(k + 1, in_[c], true);
                        else dst[r] = where(c);
                    } else {
                        const uint32_t n = where(c);
                        dst[r] = packed ? (((in_[c] & 0xFFu) << 24) | n) : n;
                    }
                }
                break;
            case I_DAG_LEAF:
                dst[0] = last ? src[0] : ptr_to(k + 1, src[0], false);
                break;
        }
    }

    const Spec& sp_;
    const std::vector<uint32_t>& in_;
    std::vector<uint8_t> seen_;
    std::vector<Item> items_;
    std::vector<uint32_t> order_;
    std::vector<uint32_t> newoff_;
    int j0_[kMaxFormatLevels] = {};
    int nlev_;
    bool ok_ = true;
};

}  // namespace

bool make_device_image(const Spec& spec, const std::vector<uint32_t>& canonical, std::vector<uint32_t>& out,
                       bool* packed, uint32_t* stage_end) {
    bool pk = false;
    Relocator r(spec, canonical);
    if (!r.run(out, pk)) {
        out.clear();
        return false;
    }
    *packed = pk;
    if (stage_end)
        for (int k = 0; k <= kStageLevels; k++) stage_end[k] = r.stage_end[k];
    return true;
}

}  // namespace vx
