// validate.cpp -- checks a word buffer against the paper's layout (Sec. 3.3)
// before it is used as a volume (vx_load): every pointer stays inside the
// buffer, octree masks are consistent with their depth (Fig. 3: valid mask,
// leaf mask set exactly at the last depth), valid children are non-empty, and
// every DF distance equals the capped L1 distance of its sub-volume
// (Table 1, Sec. 4.1).  Each node is checked once per node level it is
// reached at, so shared SVDAG nodes cost once and corrupt sharing cannot
// blow the walk up.
#include <string.h>

#include "vx_internal.hpp"

namespace vx {
namespace {

class Validator {
  public:
    Validator(const Spec& sp, const uint32_t* w, uint64_t n, BuildResult& R) : sp_(sp), w_(w), n_(n), R_(R) {
        nlev_ = (int)sp.lv.size();
        int j = 0;
        for (int k = 0; k < nlev_; k++) {
            j0_[k] = j;
            j += sp.lv[k].kind == K_SVO || sp.lv[k].kind == K_DAG ? sp.lv[k].e[0] : 1;
        }
        seen_.assign(n, 0);
    }
    int run() {
        if (n_ < 1) return fail(VX_EINVAL, "empty buffer (word 0 holds the root pointer)");
        if (w_[0] != 0) level(0, w_[0]);
        return err_;
    }

  private:
    bool bad(const char* what, uint64_t p) {
        if (!err_) err_ = fail(VX_EINVAL, "invalid buffer: %s at word %llu", what, (unsigned long long)p);
        return false;
    }
    bool in(uint64_t p, uint64_t k) { return (p != 0 && p + k <= n_) || bad("pointer out of range", p); }
    // first visit of node p at node level j?
    bool first(uint64_t p, int j) {
        const uint16_t bit = (uint16_t)(1u << j);
        if (seen_[p] & bit) return false;
        seen_[p] |= bit;
        return true;
    }
    void level(int k, uint32_t p) {
        if (err_) return;
        const Level& L = sp_.lv[k];
        const bool last = k == nlev_ - 1;
        if (L.kind == K_RAW || L.kind == K_DF) {
            const uint64_t cells = 1ull << (L.e[0] + L.e[1] + L.e[2]);
            const uint64_t wpc = L.kind == K_DF ? 2 : 1;
            if (!in(p, wpc * cells) || !first(p, j0_[k])) return;
            R_.level_words[k] += wpc * cells;
            R_.level_nodes[k]++;
            if (L.kind == K_DF) {
                std::vector<uint32_t> terms(cells), d;
                for (uint64_t i = 0; i < cells; i++) terms[i] = w_[p + 2 * i];
                l1_distance(terms.data(), L.e, (uint32_t)L.m, d);
                for (uint64_t i = 0; i < cells; i++)
                    if (w_[p + 2 * i + 1] != d[i]) { bad("DF distance differs from its definition", p + 2 * i + 1); return; }
            }
            if (last) return;
            for (uint64_t i = 0; i < cells && !err_; i++) {
                const uint32_t t = w_[p + wpc * i];
                if (t) level(k + 1, t);
            }
        } else if (L.kind == K_SVO) {
            svo(k, p, 0);
        } else {
            dag(k, p, 0);
        }
    }
    bool masks_ok(uint32_t masks, int depth, int L, uint64_t at) {
        const uint32_t valid = masks & 0xFFu, leaf = (masks >> 8) & 0xFFu;
        if ((masks >> 16) != 0 || valid == 0 || leaf != (depth == L - 1 ? valid : 0u)) return bad("inconsistent masks", at);
        return true;
    }
    void svo(int k, uint32_t p, int depth) {
        if (err_ || !in(p, 2) || !first(p, j0_[k] + depth)) return;
        const int L = sp_.lv[k].e[0];
        const bool last = k == nlev_ - 1;
        if (!masks_ok(w_[p + 1], depth, L, p + 1)) return;
        const uint32_t cnt = (uint32_t)__builtin_popcount(w_[p + 1] & 0xFFu);
        const uint32_t firstc = w_[p];
        if (!in(firstc, 2ull * cnt)) return;
        R_.level_words[k] += 2ull * cnt;
        R_.level_nodes[k] += cnt;
        if (depth == 0) { R_.level_words[k] += 2; R_.level_nodes[k]++; }
        for (uint32_t r = 0; r < cnt && !err_; r++) {
            const uint64_t c = (uint64_t)firstc + 2ull * r;
            if (depth + 1 == L) {
                if (w_[c] == 0) { bad("empty leaf", c); return; }
                if (w_[c + 1] != 0) { bad("leaf second word not 0", c + 1); return; }
                if (!last) level(k + 1, w_[c]);
            } else {
                svo(k, (uint32_t)c, depth + 1);
            }
        }
    }
    void dag(int k, uint32_t p, int depth) {
        if (err_ || !in(p, 1) || !first(p, j0_[k] + depth)) return;
        const int L = sp_.lv[k].e[0];
        const bool last = k == nlev_ - 1;
        if (!masks_ok(w_[p], depth, L, p)) return;
        const uint32_t cnt = (uint32_t)__builtin_popcount(w_[p] & 0xFFu);
        if (!in(p, 1ull + cnt)) return;
        R_.level_words[k] += 1ull + cnt;
        R_.level_nodes[k]++;
        for (uint32_t r = 0; r < cnt && !err_; r++) {
            const uint32_t cp = w_[p + 1 + r];
            if (!in(cp, 1)) return;
            if (depth + 1 == L) {
                if (first(cp, 15)) { R_.level_words[k]++; R_.level_nodes[k]++; }  // leaf words
                if (w_[cp] == 0) { bad("empty leaf", cp); return; }
                if (!last) level(k + 1, w_[cp]);
            } else {
                dag(k, cp, depth + 1);
            }
        }
    }

    const Spec& sp_;
    const uint32_t* w_;
    uint64_t n_;
    BuildResult& R_;
    int nlev_;
    int j0_[kMaxFormatLevels];
    std::vector<uint16_t> seen_;  // per word: node levels it was checked at (bit 15: SVDAG leaf word)
    int err_ = 0;
};

}  // namespace

int validate_canonical(const Spec& spec, const uint32_t* words, uint64_t n, BuildResult* stats) {
    Validator v(spec, words, n, *stats);
    return v.run();
}

}  // namespace vx
