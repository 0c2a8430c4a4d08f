// pack.cpp -- the device image of a volume.
//
// The canonical buffer follows the paper's layout (Sec. 3.3), where reaching
// an SVDAG child costs two dependent reads: the child pointer in the parent,
// then the child's masks word (and, at the last octree level, a third read:
// the leaf's terminating integer).  The packed device image keeps every
// offset of the canonical buffer and rewrites three kinds of words in place:
//   - a pointer to an SVDAG node p becomes (valid mask of p) << 24 | p;
//   - an SVDAG node's slot for a leaf child holds the leaf's terminating
//     integer itself instead of a pointer to it;
//   - word 0 (root pointer) and Raw / DF cells / SVO leaf words that point
//     at an SVDAG root follow the first rule.
// It needs every offset below 2^24 words (64 MiB); larger volumes keep the
// canonical words on the device (the kernels are told which layout they
// read).
#include <string.h>

#include <vector>

#include "vx_internal.hpp"

namespace vx {
namespace {

class Packer {
  public:
    Packer(const Spec& sp, const std::vector<uint32_t>& in, std::vector<uint32_t>& out)
        : sp_(sp), in_(in), out_(out), seen_(in.size(), 0) {
        nlev_ = (int)sp.lv.size();
    }

    bool run() {
        out_ = in_;
        if (in_[0] == 0) return true;
        out_[0] = ptr_for(0, in_[0]);
        level(0, in_[0]);
        return ok_;
    }

  private:
    // The word a parent stores for the root of level k's sub-volume at p.
    uint32_t ptr_for(int k, uint32_t p) const {
        if (sp_.lv[k].kind == K_DAG) return ((in_[p] & 0xFFu) << 24) | p;
        return p;
    }
    bool check(uint64_t p, uint64_t n) {
        if (p == 0 || p + n > in_.size()) ok_ = false;
        return ok_;
    }
    void level(int k, uint32_t p) {
        if (!ok_ || seen_[p]) return;
        seen_[p] = 1;
        const Level& L = sp_.lv[k];
        const bool last = k == nlev_ - 1;
        if (L.kind == K_RAW || L.kind == K_DF) {
            const uint64_t cells = 1ull << (L.e[0] + L.e[1] + L.e[2]);
            const uint64_t wpc = L.kind == K_DF ? 2 : 1;  // DF: {terminating integer, distance}
            if (!check(p, wpc * cells) || last) return;
            for (uint64_t i = 0; i < cells; i++) {
                const uint32_t w = in_[p + wpc * i];
                if (!w) continue;
                level(k + 1, w);
                out_[p + wpc * i] = ptr_for(k + 1, w);
            }
        } else if (L.kind == K_SVO) {
            svo(k, p, 0);
        } else {
            dag(k, p, 0);
        }
    }
    void svo(int k, uint32_t p, int depth) {
        if (!check(p, 2)) return;
        const int L = sp_.lv[k].e[0];
        const bool last = k == nlev_ - 1;
        const uint32_t first = in_[p], valid = in_[p + 1] & 0xFFu;
        const uint32_t cnt = __builtin_popcount(valid);
        if (!check(first, 2ull * cnt)) return;
        for (uint32_t r = 0; r < cnt; r++) {
            const uint32_t c = first + 2 * r;
            if (depth + 1 == L) {
                if (last) continue;
                const uint32_t term = in_[c];
                level(k + 1, term);
                out_[c] = ptr_for(k + 1, term);
            } else {
                svo(k, c, depth + 1);
            }
        }
    }
    void dag(int k, uint32_t p, int depth) {
        if (!check(p, 1)) return;
        if (depth > 0) {  // roots are marked by level()
            if (seen_[p]) return;
            seen_[p] = 1;
        }
        const int L = sp_.lv[k].e[0];
        const bool last = k == nlev_ - 1;
        const uint32_t valid = in_[p] & 0xFFu;
        const uint32_t cnt = __builtin_popcount(valid);
        if (!check(p, 1ull + cnt)) return;
        for (uint32_t r = 0; r < cnt; r++) {
            const uint32_t slot = p + 1 + r;
            const uint32_t c = in_[slot];
            if (!check(c, 1)) return;
            if (depth + 1 == L) {
                const uint32_t term = in_[c];
                if (last) {
                    out_[slot] = term;
                } else {
                    level(k + 1, term);
                    out_[slot] = ptr_for(k + 1, term);
                }
            } else {
                dag(k, c, depth + 1);
                out_[slot] = ((in_[c] & 0xFFu) << 24) | c;
            }
        }
    }

    const Spec& sp_;
    const std::vector<uint32_t>& in_;
    std::vector<uint32_t>& out_;
    std::vector<uint8_t> seen_;
    int nlev_;
    bool ok_ = true;
};

}  // namespace

bool pack_device_image(const Spec& spec, const std::vector<uint32_t>& canonical, std::vector<uint32_t>& out) {
    if (canonical.size() >= (1u << 24)) return false;
    bool any_dag = false;
    for (const Level& L : spec.lv) any_dag |= L.kind == K_DAG;
    if (!any_dag) return false;  // nothing to rewrite
    Packer p(spec, canonical, out);
    return p.run();
}

}  // namespace vx
