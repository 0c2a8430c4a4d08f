// build.cpp -- host construction of a hybrid format in the paper's word-buffer
// layout, and its inverse (decoding a cube of voxels).
//
// Construction follows Sec. 4.1 and Fig. 4 (construct): the function of level
// k maps the lower corner of a sub-volume to its data; for every child cell it
// asks level k+1 for the child's sub-volume, writes it to the buffer unless
// it is empty (then the child pointer is 0), and stores the pointer.  Children
// are visited in Morton order (Sec. 5, Fig. 5), so every pointer refers to
// words already written, and the root function writes the root sub-volume
// last and its pointer into word 0 (Sec. 4.1).
//
// Layout (Sec. 3.3, Fig. 3):
//   Raw R(W,H,D): 2^(W+H+D) terminating integers, cell (x,y,z) at
//     x + (y << W) + (z << (W+H)).
//   DF D(W,H,D,M): the same cells, two interleaved words each: the
//     terminating integer and the L1 distance (in cells) to the nearest
//     non-empty cell of the sub-volume, capped at M; computed once all the
//     children are recorded (Sec. 4.1).
//   SVO S(L): 2-word nodes {first-child pointer | terminating integer,
//     valid | leaf << 8}; a node's valid children are written contiguously,
//     2 words each, in child-index order (i = x | y << 1 | z << 2), when the
//     node is formed; leaf children (depth L) are {terminating integer, 0}.
//     The root node is the sub-volume's data.  This is the bottom-up
//     construction of Baert et al. that the paper uses, written as a
//     post-order recursion: a node is formed right after its last child,
//     exactly when the queue-based form would form it.
//   SVDAG G(L): nodes {valid | leaf << 8, one pointer per valid child};
//     leaf nodes are one terminating-integer word.  When a node is formed,
//     each child is looked up in the de-duplication map and written only if
//     absent (Sec. 4.1); the map is per sub-volume, or shared by the whole
//     level with VX_DEDUP_WHOLE_LEVEL (Sec. 4.3).
// A terminating integer is the word offset of the next level's sub-volume,
// or the voxel's RGBA at the last level; 0 is empty (Sec. 3.3).
#include <omp.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <unordered_map>

#include "vx_internal.hpp"

namespace vx {

// ---------------------------------------------------------------------------
// Dense host grid with an occupancy pyramid for empty-cube tests.
// ---------------------------------------------------------------------------
namespace {

class DenseSource final : public VoxelSource {
  public:
    // Either RGBA words (w) or 8-bit palette indices (w8 + palette).
    DenseSource(const uint32_t* w, const uint8_t* w8, const uint32_t* pal, const int ld[3])
        : w_(w), w8_(w8), pal_(pal) {
        for (int i = 0; i < 3; i++) { ld_[i] = ld[i]; n_[i] = (int64_t)1 << ld[i]; }
        levels_ = std::max(ld[0], std::max(ld[1], ld[2])) + 1;
        pyr_.resize(levels_);
        for (int m = 0; m < levels_; m++) {
            for (int i = 0; i < 3; i++) pn_[m][i] = std::max<int64_t>(1, n_[i] >> m);
            pyr_[m].assign((size_t)((pn_[m][0] * pn_[m][1] * pn_[m][2] + 63) / 64), 0ull);
        }
        const int64_t total = n_[0] * n_[1] * n_[2];
        const int64_t words = (total + 63) / 64;
        // level 0: one bit per voxel, 64 voxels per word (parallel over words)
#pragma omp parallel for schedule(static)
        for (int64_t wi = 0; wi < words; wi++) {
            uint64_t bits = 0;
            const int64_t i0 = wi * 64, i1 = std::min<int64_t>(i0 + 64, total);
            for (int64_t i = i0; i < i1; i++)
                if (w_ ? w_[i] != 0 : pal_[w8_[i]] != 0) bits |= 1ull << (i - i0);
            pyr_[0][(size_t)wi] = bits;
        }
        // coarser levels: OR of 2x2x2 children (parallel over output z-slabs
        // of 32 cells; each output word belongs to one slab when x-rows are
        // a multiple of 64 cells, else serial)
        for (int m = 1; m < levels_; m++) {
            const int64_t X = pn_[m][0], Y = pn_[m][1], Z = pn_[m][2];
            const bool par = (X * Y) % 64 == 0;
#pragma omp parallel for schedule(static) if (par)
            for (int64_t z = 0; z < Z; z++)
                for (int64_t y = 0; y < Y; y++)
                    for (int64_t x = 0; x < X; x++) {
                        bool any = false;
                        for (int dz = 0; dz < 2 && !any; dz++)
                            for (int dy = 0; dy < 2 && !any; dy++)
                                for (int dx = 0; dx < 2 && !any; dx++) {
                                    const int64_t cx = 2 * x + dx, cy = 2 * y + dy, cz = 2 * z + dz;
                                    if (cx < pn_[m - 1][0] && cy < pn_[m - 1][1] && cz < pn_[m - 1][2])
                                        any = bit(m - 1, cx, cy, cz);
                                }
                        if (any) set(m, x, y, z);
                    }
        }
    }
    bool thread_safe() const override { return true; }
    bool empty(int64_t x0, int64_t y0, int64_t z0, int s) override {
        if (s >= levels_) s = levels_ - 1;
        return !bit(s, x0 >> s, y0 >> s, z0 >> s);
    }
    int block(int64_t x0, int64_t y0, int64_t z0, int s, uint32_t* out) override {
        const int64_t side = (int64_t)1 << s;
        for (int64_t z = 0; z < side; z++)
            for (int64_t y = 0; y < side; y++) {
                const int64_t row = x0 + n_[0] * ((y0 + y) + n_[1] * (z0 + z));
                uint32_t* o = out + side * (y + side * z);
                if (w_) memcpy(o, w_ + row, sizeof(uint32_t) * side);
                else
                    for (int64_t x = 0; x < side; x++) o[x] = pal_[w8_[row + x]];
            }
        return 0;
    }

  private:
    bool bit(int m, int64_t x, int64_t y, int64_t z) const {
        int64_t i = x + pn_[m][0] * (y + pn_[m][1] * z);
        return (pyr_[m][(size_t)(i >> 6)] >> (i & 63)) & 1ull;
    }
    void set(int m, int64_t x, int64_t y, int64_t z) {
        int64_t i = x + pn_[m][0] * (y + pn_[m][1] * z);
        pyr_[m][(size_t)(i >> 6)] |= 1ull << (i & 63);
    }
    const uint32_t* w_;
    const uint8_t* w8_;
    const uint32_t* pal_;
    int ld_[3];
    int64_t n_[3];
    int levels_;
    int64_t pn_[kMaxLog2Dim + 2][3];
    std::vector<std::vector<uint64_t>> pyr_;
};

// ---------------------------------------------------------------------------
// Grid produced brick by brick by a callback (the lazy voxelizer of Sec. 5):
// cubes of side 2^kBrick are fetched on demand, their emptiness remembered,
// and the last few kept in an LRU cache.
// ---------------------------------------------------------------------------
class BrickSource final : public VoxelSource {
  public:
    explicit BrickSource(const vx_grid* g) : g_(*g) {
        int mn = 64;
        for (int i = 0; i < 3; i++) { ld_[i] = (int)g->log2_dim[i]; mn = std::min(mn, ld_[i]); }
        bl_ = std::min(6, mn);
        for (int i = 0; i < 3; i++) nb_[i] = (int64_t)1 << (ld_[i] - bl_);
        known_.assign((size_t)(nb_[0] * nb_[1] * nb_[2]), 0);
    }
    bool empty(int64_t x0, int64_t y0, int64_t z0, int s) override {
        if (g_.block_empty && g_.block_empty(g_.user, (uint32_t)x0, (uint32_t)y0, (uint32_t)z0, (uint32_t)s)) return true;
        if (s >= bl_) {
            const int64_t k = (int64_t)1 << (s - bl_);
            for (int64_t bz = z0 >> bl_; bz < (z0 >> bl_) + k; bz++)
                for (int64_t by = y0 >> bl_; by < (y0 >> bl_) + k; by++)
                    for (int64_t bx = x0 >> bl_; bx < (x0 >> bl_) + k; bx++)
                        if (!brick_empty(bx, by, bz)) return false;
            return true;
        }
        if (brick_empty(x0 >> bl_, y0 >> bl_, z0 >> bl_)) return true;
        const Brick* b = fetch(x0 >> bl_, y0 >> bl_, z0 >> bl_);
        if (!b) return false;
        // the brick's occupancy pyramid: level s has (2^bl / 2^s)^3 cells
        const int64_t bs = (int64_t)1 << bl_;
        const int64_t m = bs >> s;
        const int64_t i = ((x0 & (bs - 1)) >> s) + m * (((y0 & (bs - 1)) >> s) + m * ((z0 & (bs - 1)) >> s));
        return !((b->pyr[s][(size_t)(i >> 6)] >> (i & 63)) & 1ull);
    }
    int block(int64_t x0, int64_t y0, int64_t z0, int s, uint32_t* out) override {
        const int64_t side = (int64_t)1 << s;
        if (s >= bl_) {
            // several bricks: copy each
            const int64_t bs = (int64_t)1 << bl_;
            for (int64_t bz = 0; bz < side; bz += bs)
                for (int64_t by = 0; by < side; by += bs)
                    for (int64_t bx = 0; bx < side; bx += bs) {
                        const Brick* b = fetch((x0 + bx) >> bl_, (y0 + by) >> bl_, (z0 + bz) >> bl_);
                        if (!b) return VX_EINVAL;
                        for (int64_t z = 0; z < bs; z++)
                            for (int64_t y = 0; y < bs; y++)
                                memcpy(out + (bx + side * ((by + y) + side * (bz + z))), b->w.data() + bs * (y + bs * z),
                                       sizeof(uint32_t) * bs);
                    }
            return 0;
        }
        const Brick* b = fetch(x0 >> bl_, y0 >> bl_, z0 >> bl_);
        if (!b) return VX_EINVAL;
        const int64_t bs = (int64_t)1 << bl_;
        const int64_t ox = x0 & (bs - 1), oy = y0 & (bs - 1), oz = z0 & (bs - 1);
        for (int64_t z = 0; z < side; z++)
            for (int64_t y = 0; y < side; y++)
                memcpy(out + side * (y + side * z), b->w.data() + (ox + bs * ((oy + y) + bs * (oz + z))),
                       sizeof(uint32_t) * side);
        return 0;
    }
    int error() const { return err_; }

  private:
    struct Brick {
        int64_t key;
        std::vector<uint32_t> w;
        std::vector<uint64_t> pyr[7];  // occupancy bits per level (cells of side 2^level)
        uint64_t stamp;
    };
    void build_pyramid(Brick& b) {
        const int64_t bs = (int64_t)1 << bl_;
        for (int l = 0; l <= bl_; l++) {
            const int64_t m = bs >> l;
            b.pyr[l].assign((size_t)((m * m * m + 63) / 64), 0ull);
        }
        for (int64_t i = 0; i < bs * bs * bs; i++)
            if (b.w[(size_t)i]) b.pyr[0][(size_t)(i >> 6)] |= 1ull << (i & 63);
        for (int l = 1; l <= bl_; l++) {
            const int64_t mp = bs >> (l - 1), m = bs >> l;
            for (int64_t z = 0; z < mp; z++)
                for (int64_t y = 0; y < mp; y++)
                    for (int64_t x = 0; x < mp; x++) {
                        const int64_t i = x + mp * (y + mp * z);
                        if ((b.pyr[l - 1][(size_t)(i >> 6)] >> (i & 63)) & 1ull) {
                            const int64_t j = (x >> 1) + m * ((y >> 1) + m * (z >> 1));
                            b.pyr[l][(size_t)(j >> 6)] |= 1ull << (j & 63);
                        }
                    }
        }
    }
    bool brick_empty(int64_t bx, int64_t by, int64_t bz) {
        size_t i = (size_t)(bx + nb_[0] * (by + nb_[1] * bz));
        if (!known_[i]) fetch(bx, by, bz);
        return known_[i] == 1;
    }
    const Brick* fetch(int64_t bx, int64_t by, int64_t bz) {
        const int64_t key = bx + nb_[0] * (by + nb_[1] * bz);
        for (auto& b : cache_)
            if (b.key == key) { b.stamp = ++clock_; return &b; }
        Brick* slot = nullptr;
        if (cache_.size() < kCache) {
            cache_.push_back(Brick{});
            slot = &cache_.back();
        } else {
            slot = &*std::min_element(cache_.begin(), cache_.end(),
                                      [](const Brick& a, const Brick& b) { return a.stamp < b.stamp; });
        }
        const int64_t bs = (int64_t)1 << bl_;
        slot->w.resize((size_t)(bs * bs * bs));
        slot->key = key;
        slot->stamp = ++clock_;
        if (g_.fill_brick(g_.user, (uint32_t)(bx * bs), (uint32_t)(by * bs), (uint32_t)(bz * bs), (uint32_t)bl_,
                          slot->w.data()) != 0) {
            err_ = VX_EINVAL;
            std::fill(slot->w.begin(), slot->w.end(), 0u);
        }
        build_pyramid(*slot);
        const bool any = (slot->pyr[bl_][0] & 1ull) != 0;
        known_[(size_t)key] = any ? 2 : 1;
        return slot;
    }
    static constexpr size_t kCache = 64;
    vx_grid g_;
    int ld_[3];
    int bl_;
    int64_t nb_[3];
    std::vector<uint8_t> known_;  // 0 unknown, 1 empty, 2 occupied
    std::vector<Brick> cache_;
    uint64_t clock_ = 0;
    int err_ = 0;
};

// ---------------------------------------------------------------------------
// Builder
// ---------------------------------------------------------------------------
struct NodeKey {
    uint32_t n;
    uint32_t w[9];
    bool operator==(const NodeKey& o) const {
        if (n != o.n) return false;
        for (uint32_t i = 0; i < n; i++)
            if (w[i] != o.w[i]) return false;
        return true;
    }
};
struct NodeKeyHash {
    size_t operator()(const NodeKey& k) const {
        uint64_t h = 0x9E3779B97F4A7C15ull ^ k.n;
        for (uint32_t i = 0; i < k.n; i++) {
            h ^= k.w[i];
            h *= 0xBF58476D1CE4E5B9ull;
            h ^= h >> 29;
        }
        return (size_t)h;
    }
};

// What a write holds, for relocating it when fragments are merged.
enum WriteTag : uint8_t {
    T_RAW = 0,        // Raw array (pointers to level k+1 unless k is last)
    T_DF,             // DF array {terminating integer, distance} per cell
    T_SVO_ROOT,       // SVO root node {children list, masks}
    T_DAG_ROOT,       // SVDAG root node (not de-duplicated)
    T_SVO_LIST,       // contiguous internal SVO nodes
    T_SVO_LIST_LEAF,  // contiguous leaf SVO nodes {terminating integer, 0}
    T_DAG_CHILD,      // de-duplicated SVDAG node (1 word = leaf)
};
struct WriteRec {
    uint32_t off, n;
    uint8_t tag, level;
};

}  // namespace

// L1 distance transform of a W x H x D grid of cells, capped at M: d = 0 on
// non-empty cells, else min(M, distance to the nearest non-empty cell).  The
// L1 metric separates by axis, so a forward and a backward sweep along x,
// then y, then z (each d = min(d, neighbour + 1)) give the exact distances.
void l1_distance(const uint32_t* terms, const int e[3], uint32_t M, std::vector<uint32_t>& d) {
    const int64_t n[3] = {(int64_t)1 << e[0], (int64_t)1 << e[1], (int64_t)1 << e[2]};
    const int64_t stride[3] = {1, n[0], n[0] * n[1]};
    const int64_t cells = n[0] * n[1] * n[2];
    d.resize((size_t)cells);
    for (int64_t i = 0; i < cells; i++) d[(size_t)i] = terms[i] ? 0u : M;
    for (int a = 0; a < 3; a++) {
        if (n[a] == 1) continue;
        const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
        for (int64_t u = 0; u < n[b]; u++)
            for (int64_t v = 0; v < n[c]; v++) {
                uint32_t* row = d.data() + u * stride[b] + v * stride[c];
                const int64_t st = stride[a];
                for (int64_t i = 1; i < n[a]; i++) row[i * st] = std::min(row[i * st], row[(i - 1) * st] + 1);
                for (int64_t i = n[a] - 2; i >= 0; i--) row[i * st] = std::min(row[i * st], row[(i + 1) * st] + 1);
            }
    }
}

namespace {

// Interleaves terminating integers and distances into a DF sub-volume.
void df_words(const std::vector<uint32_t>& terms, const int e[3], uint32_t M, std::vector<uint32_t>& out) {
    std::vector<uint32_t> d;
    l1_distance(terms.data(), e, M, d);
    out.resize(2 * terms.size());
    for (size_t i = 0; i < terms.size(); i++) { out[2 * i] = terms[i]; out[2 * i + 1] = d[i]; }
}

class Builder {
  public:
    Builder(const Spec& sp, VoxelSource& src, int scope, BuildResult& R) : sp_(sp), src_(src), scope_(scope), R_(R) {
        nlev_ = (int)sp.lv.size();
        int acc = 0;
        for (int k = nlev_ - 1; k >= 0; k--) {
            s_[k] = acc;  // cell side of level k (cubic below the top level)
            acc += sp.lv[k].e[0];
        }
        maps_.resize(nlev_);
        leaf_cache_.assign(nlev_, std::vector<LeafSlot>(1u << kLeafCacheBits));
        map_gen_.assign(nlev_, 1u);
        for (int i = 0; i < 3; i++) cb_[i] = std::min(5, sp.ldim[i]);
        cside_ = std::min(cb_[0], std::min(cb_[1], cb_[2]));
        cache_.resize((size_t)1 << (3 * cside_));
    }

    int run() {
        R_.words.assign(1, 0u);
        std::vector<uint32_t> data;
        const int64_t lo[3] = {0, 0, 0};
        if (construct(0, lo, data)) {
            uint32_t p = write(0, data.data(), data.size(), root_tag(0));
            if (!err_) R_.words[0] = p;
        }
        return err_;
    }

    // Parallel build for a Raw top level over a thread-safe source: every
    // top cell's sub-volume is built as a fragment (own buffer, own maps,
    // write log) on its own thread; the fragments are then appended in the
    // Morton order of their cells, pointers relocated and SVDAG nodes looked
    // up in this builder's maps, so the buffer equals the sequential one.
    int run_parallel(int threads) {
        const Level& L0 = sp_.lv[0];
        const uint64_t cells = 1ull << (L0.e[0] + L0.e[1] + L0.e[2]);
        struct Frag {
            std::vector<uint32_t> words;
            std::vector<WriteRec> log;
            uint32_t root = 0;
            uint64_t occupied = 0;
            int err = 0;
            std::string msg;
        };
        std::vector<Frag> frags(cells);
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
        for (int64_t m = 0; m < (int64_t)cells; m++) {
            uint32_t c[3];
            morton_decode((uint64_t)m, L0.e, c);
            const int64_t lo[3] = {(int64_t)c[0] << s_[0], (int64_t)c[1] << s_[0], (int64_t)c[2] << s_[0]};
            Frag& F = frags[(size_t)m];
            if (src_.empty(lo[0], lo[1], lo[2], s_[0])) continue;
            BuildResult local;
            local.words.assign(1, 0u);  // offsets start at 1: 0 stays "empty"
            Builder b(sp_, src_, scope_, local);
            b.log_ = &F.log;
            std::vector<uint32_t> data;
            if (b.construct(1, lo, data)) F.root = b.write(1, data.data(), data.size(), b.root_tag(1));
            F.err = b.err_;
            if (F.err) F.msg = vx_last_error();
            F.words.swap(local.words);
            F.occupied = local.occupied;
        }
        R_.words.assign(1, 0u);
        std::vector<uint32_t> top((size_t)cells, 0u);
        bool any = false;
        for (uint64_t m = 0; m < cells && !err_; m++) {
            Frag& F = frags[(size_t)m];
            if (F.err) return fail(F.err, "%s", F.msg.c_str());
            R_.occupied += F.occupied;
            if (!F.root) continue;
            uint32_t c[3];
            morton_decode(m, L0.e, c);
            top[(size_t)(c[0] + ((uint64_t)c[1] << L0.e[0]) + ((uint64_t)c[2] << (L0.e[0] + L0.e[1])))] = merge(F.words, F.log, F.root);
            any = true;
            std::vector<uint32_t>().swap(F.words);
            std::vector<WriteRec>().swap(F.log);
        }
        if (any && !err_) {
            if (L0.kind == K_DF) {
                std::vector<uint32_t> df;
                df_words(top, L0.e, (uint32_t)L0.m, df);
                R_.words[0] = write(0, df.data(), df.size(), T_DF);
            } else {
                R_.words[0] = write(0, top.data(), top.size(), T_RAW);
            }
            R_.level_nodes[0]++;
        }
        return err_;
    }

  private:
    uint8_t root_tag(int k) const {
        const int kind = sp_.lv[k].kind;
        return kind == K_RAW ? T_RAW : (kind == K_DF ? T_DF : (kind == K_SVO ? T_SVO_ROOT : T_DAG_ROOT));
    }

    uint32_t write(int k, const uint32_t* w, size_t n, uint8_t tag) {
        if (R_.words.size() + n > 0xFFFFFFFFull) {
            err_ = fail(VX_ETOOBIG, "format buffer exceeds 2^32 words (16 GiB, Sec. 3.3)");
            return 0;
        }
        uint32_t off = (uint32_t)R_.words.size();
        R_.words.insert(R_.words.end(), w, w + n);
        R_.level_words[k] += n;
        if (log_) log_->push_back(WriteRec{off, (uint32_t)n, tag, (uint8_t)k});
        return off;
    }

    // Appends one fragment; returns the global offset of its root.
    uint32_t merge(const std::vector<uint32_t>& fw, const std::vector<WriteRec>& log, uint32_t root) {
        std::vector<uint32_t> reloc(fw.size(), 0u);
        std::vector<uint32_t> tmp;
        for (const WriteRec& r : log) {
            if (err_) return 0;
            const int k = r.level;
            const bool last = k == nlev_ - 1;
            tmp.assign(fw.begin() + r.off, fw.begin() + r.off + r.n);
            switch (r.tag) {
                case T_RAW:
                    if (!last)
                        for (uint32_t& x : tmp)
                            if (x) x = reloc[x];
                    break;
                case T_DF:
                    if (!last)
                        for (size_t i = 0; i < tmp.size(); i += 2)
                            if (tmp[i]) tmp[i] = reloc[tmp[i]];
                    break;
                case T_SVO_ROOT:
                case T_SVO_LIST:
                    for (size_t i = 0; i < tmp.size(); i += 2) tmp[i] = reloc[tmp[i]];
                    break;
                case T_SVO_LIST_LEAF:
                    if (!last)
                        for (size_t i = 0; i < tmp.size(); i += 2) tmp[i] = reloc[tmp[i]];
                    break;
                default:  // SVDAG node: a leaf word, or masks + child pointers
                    if (tmp.size() == 1) {
                        if (!last) tmp[0] = reloc[tmp[0]];
                    } else {
                        for (size_t i = 1; i < tmp.size(); i++) tmp[i] = reloc[tmp[i]];
                    }
            }
            uint32_t g;
            if (r.tag == T_DAG_CHILD && scope_ == VX_DEDUP_WHOLE_LEVEL) {
                NodeKey key;
                key.n = (uint32_t)tmp.size();
                for (uint32_t i = 0; i < key.n; i++) key.w[i] = tmp[i];
                auto it = maps_[k].find(key);
                if (it != maps_[k].end()) {
                    g = it->second;
                } else {
                    g = write(k, tmp.data(), tmp.size(), r.tag);
                    R_.level_nodes[k]++;
                    maps_[k].emplace(key, g);
                }
            } else {
                g = write(k, tmp.data(), tmp.size(), r.tag);
                if (r.tag == T_SVO_LIST || r.tag == T_SVO_LIST_LEAF) R_.level_nodes[k] += r.n / 2;
                else R_.level_nodes[k]++;
            }
            reloc[r.off] = g;
        }
        return reloc[root];
    }

    uint32_t voxel(const int64_t v[3]) {
        const int64_t m = (int64_t)1 << cside_;
        const int64_t c[3] = {v[0] & ~(m - 1), v[1] & ~(m - 1), v[2] & ~(m - 1)};
        if (!cache_valid_ || c[0] != corner_[0] || c[1] != corner_[1] || c[2] != corner_[2]) {
            if (src_.block(c[0], c[1], c[2], cside_, cache_.data()) != 0)
                err_ = fail(VX_EINVAL, "voxel source failed for brick at (%lld,%lld,%lld)", (long long)c[0],
                            (long long)c[1], (long long)c[2]);
            corner_[0] = c[0]; corner_[1] = c[1]; corner_[2] = c[2];
            cache_valid_ = true;
        }
        uint32_t w = cache_[(size_t)((v[0] - c[0]) + m * ((v[1] - c[1]) + m * (v[2] - c[2])))];
        if (w) R_.occupied++;
        return w;
    }

    // Terminating integer of the level-k cell with lower corner lo.
    uint32_t cell_term(int k, const int64_t lo[3]) {
        if (k == nlev_ - 1) return voxel(lo);
        if (src_.empty(lo[0], lo[1], lo[2], s_[k])) return 0;
        std::vector<uint32_t> data;
        if (!construct(k + 1, lo, data)) return 0;
        return write(k + 1, data.data(), data.size(), root_tag(k + 1));
    }

    // Sub-volume of level k at lo; false if it is empty.
    bool construct(int k, const int64_t lo[3], std::vector<uint32_t>& data) {
        if (err_) return false;
        const Level& L = sp_.lv[k];
        if (L.kind == K_RAW || L.kind == K_DF) {
            const uint64_t cells = 1ull << (L.e[0] + L.e[1] + L.e[2]);
            data.assign((size_t)cells, 0u);
            bool any = false;
            for (uint64_t m = 0; m < cells && !err_; m++) {
                uint32_t c[3];
                morton_decode(m, L.e, c);
                const int64_t cl[3] = {lo[0] + ((int64_t)c[0] << s_[k]), lo[1] + ((int64_t)c[1] << s_[k]),
                                       lo[2] + ((int64_t)c[2] << s_[k])};
                uint32_t t = cell_term(k, cl);
                data[(size_t)(c[0] + ((uint64_t)c[1] << L.e[0]) + ((uint64_t)c[2] << (L.e[0] + L.e[1])))] = t;
                any |= t != 0;
            }
            if (any) R_.level_nodes[k]++;
            if (any && L.kind == K_DF) {
                std::vector<uint32_t> df;
                df_words(data, L.e, (uint32_t)L.m, df);
                data.swap(df);
            }
            return any && !err_;
        }
        if (L.kind == K_DAG && scope_ == VX_DEDUP_PER_SUBVOLUME) {
            maps_[k].clear();
            map_gen_[k]++;  // invalidates the leaf cache of this level
        }
        NodeKey root;
        bool ok = (L.kind == K_SVO) ? svo_node(k, lo, 0, root) : dag_node(k, lo, 0, root);
        if (!ok || err_) return false;
        data.assign(root.w, root.w + root.n);
        R_.level_nodes[k]++;
        return true;
    }

    // Octree node of format level k at depth `depth` (0 = root, L = leaf).
    bool svo_node(int k, const int64_t lo[3], int depth, NodeKey& out) {
        const int L = sp_.lv[k].e[0];
        const int side = s_[k] + L - depth;
        if (depth == L) {
            uint32_t t = cell_term(k, lo);
            if (!t) return false;
            out.n = 2; out.w[0] = t; out.w[1] = 0;
            return true;
        }
        if (side > 0 && src_.empty(lo[0], lo[1], lo[2], side)) return false;
        NodeKey ch[8];
        uint32_t valid = 0;
        for (int i = 0; i < 8 && !err_; i++) {
            const int64_t h = (int64_t)1 << (side - 1);
            const int64_t cl[3] = {lo[0] + (i & 1) * h, lo[1] + ((i >> 1) & 1) * h, lo[2] + ((i >> 2) & 1) * h};
            if (svo_node(k, cl, depth + 1, ch[i])) valid |= 1u << i;
        }
        if (!valid || err_) return false;
        uint32_t buf[16];
        uint32_t n = 0;
        for (int i = 0; i < 8; i++)
            if ((valid >> i) & 1u) { buf[n++] = ch[i].w[0]; buf[n++] = ch[i].w[1]; }
        const uint32_t first = write(k, buf, n, (depth + 1 == L) ? T_SVO_LIST_LEAF : T_SVO_LIST);
        R_.level_nodes[k] += n / 2;
        const uint32_t leaf = (depth + 1 == L) ? valid : 0u;
        out.n = 2; out.w[0] = first; out.w[1] = valid | (leaf << 8);
        return true;
    }

    bool dag_node(int k, const int64_t lo[3], int depth, NodeKey& out) {
        const int L = sp_.lv[k].e[0];
        const int side = s_[k] + L - depth;
        if (depth == L) {
            uint32_t t = cell_term(k, lo);
            if (!t) return false;
            out.n = 1; out.w[0] = t;
            return true;
        }
        if (side > 0 && src_.empty(lo[0], lo[1], lo[2], side)) return false;
        NodeKey ch[8];
        uint32_t valid = 0;
        for (int i = 0; i < 8 && !err_; i++) {
            const int64_t h = (int64_t)1 << (side - 1);
            const int64_t cl[3] = {lo[0] + (i & 1) * h, lo[1] + ((i >> 1) & 1) * h, lo[2] + ((i >> 2) & 1) * h};
            if (dag_node(k, cl, depth + 1, ch[i])) valid |= 1u << i;
        }
        if (!valid || err_) return false;
        const uint32_t leaf = (depth + 1 == L) ? valid : 0u;
        out.n = 1;
        out.w[0] = valid | (leaf << 8);
        auto& map = maps_[k];
        for (int i = 0; i < 8; i++) {
            if (!((valid >> i) & 1u)) continue;
            uint32_t p;
            // one-word leaf nodes repeat a few colours: a direct-mapped cache
            // in front of the map (same results, fewer hash-map probes)
            if (ch[i].n == 1) {
                LeafSlot& ls = leaf_cache_[k][(ch[i].w[0] * 2654435761u) >> (32 - kLeafCacheBits)];
                if (ls.gen == map_gen_[k] && ls.valid && ls.term == ch[i].w[0]) {
                    out.w[out.n++] = ls.ptr;
                    continue;
                }
                auto it = map.find(ch[i]);
                if (it != map.end()) {
                    p = it->second;
                } else {
                    p = write(k, ch[i].w, ch[i].n, T_DAG_CHILD);
                    R_.level_nodes[k]++;
                    map.emplace(ch[i], p);
                }
                ls.gen = map_gen_[k];
                ls.valid = true;
                ls.term = ch[i].w[0];
                ls.ptr = p;
                out.w[out.n++] = p;
                continue;
            }
            auto it = map.find(ch[i]);
            if (it != map.end()) {
                p = it->second;
            } else {
                p = write(k, ch[i].w, ch[i].n, T_DAG_CHILD);
                R_.level_nodes[k]++;
                map.emplace(ch[i], p);
            }
            out.w[out.n++] = p;
        }
        return true;
    }

    const Spec& sp_;
    VoxelSource& src_;
    int scope_;
    BuildResult& R_;
    int nlev_;
    int s_[kMaxFormatLevels];
    std::vector<std::unordered_map<NodeKey, uint32_t, NodeKeyHash>> maps_;
    static constexpr int kLeafCacheBits = 8;
    struct LeafSlot {
        uint32_t gen = 0, term = 0, ptr = 0;
        bool valid = false;
    };
    std::vector<std::vector<LeafSlot>> leaf_cache_;
    std::vector<uint32_t> map_gen_;
    int cb_[3];
    int cside_;
    std::vector<uint32_t> cache_;
    int64_t corner_[3] = {0, 0, 0};
    bool cache_valid_ = false;
    int err_ = 0;
    std::vector<WriteRec>* log_ = nullptr;
};

// ---------------------------------------------------------------------------
// Decoder: walks the buffer like the intersection functions do, visiting only
// children that overlap the requested cube.
// ---------------------------------------------------------------------------
class Decoder {
  public:
    Decoder(const Spec& sp, const uint32_t* w, uint64_t nw, const int64_t c0[3], int log2s, uint32_t* out)
        : sp_(sp), w_(w), nw_(nw), out_(out) {
        nlev_ = (int)sp.lv.size();
        int acc = 0;
        for (int k = nlev_ - 1; k >= 0; k--) { s_[k] = acc; acc += sp.lv[k].e[0]; }
        side_ = (int64_t)1 << log2s;
        for (int i = 0; i < 3; i++) c0_[i] = c0[i];
    }
    int run() {
        if (nw_ < 1) return fail(VX_EINVAL, "empty buffer");
        if (w_[0] == 0) return VX_OK;
        const int64_t lo[3] = {0, 0, 0};
        level(0, w_[0], lo);
        return err_;
    }

  private:
    bool overlaps(const int64_t lo[3], int64_t size) const {
        for (int i = 0; i < 3; i++)
            if (lo[i] + size <= c0_[i] || lo[i] >= c0_[i] + side_) return false;
        return true;
    }
    bool in(uint64_t p, uint64_t n) {
        if (p == 0 || p + n > nw_) { err_ = fail(VX_EINVAL, "pointer %llu out of range", (unsigned long long)p); return false; }
        return true;
    }
    void emit(int k, uint32_t term, const int64_t lo[3]) {
        if (k == nlev_ - 1) {
            out_[(size_t)((lo[0] - c0_[0]) + side_ * ((lo[1] - c0_[1]) + side_ * (lo[2] - c0_[2])))] = term;
        } else {
            level(k + 1, term, lo);
        }
    }
    void level(int k, uint32_t p, const int64_t lo[3]) {
        if (err_) return;
        const Level& L = sp_.lv[k];
        const int64_t cs = (int64_t)1 << s_[k];
        if (L.kind == K_RAW || L.kind == K_DF) {
            const uint64_t cells = 1ull << (L.e[0] + L.e[1] + L.e[2]);
            const uint64_t wpc = L.kind == K_DF ? 2 : 1;  // words per cell
            if (!in(p, wpc * cells)) return;
            for (int64_t z = 0; z < (1 << L.e[2]); z++)
                for (int64_t y = 0; y < (1 << L.e[1]); y++)
                    for (int64_t x = 0; x < (1 << L.e[0]); x++) {
                        const int64_t cl[3] = {lo[0] + x * cs, lo[1] + y * cs, lo[2] + z * cs};
                        if (!overlaps(cl, cs)) continue;
                        uint32_t t = w_[p + wpc * (x + (y << L.e[0]) + (z << (L.e[0] + L.e[1])))];
                        if (t) emit(k, t, cl);
                        if (err_) return;
                    }
        } else {
            node(k, p, 0, lo);
        }
    }
    void node(int k, uint32_t p, int depth, const int64_t lo[3]) {
        if (err_) return;
        const Level& L = sp_.lv[k];
        const bool svo = L.kind == K_SVO;
        if (!in(p, svo ? 2 : 1)) return;
        const uint32_t masks = svo ? w_[p + 1] : w_[p];
        const uint32_t valid = masks & 0xFFu;
        const int64_t half = (int64_t)1 << (s_[k] + L.e[0] - depth - 1);
        uint32_t rank = 0;
        for (int i = 0; i < 8; i++) {
            if (!((valid >> i) & 1u)) continue;
            const uint32_t r = rank++;
            const int64_t cl[3] = {lo[0] + (i & 1) * half, lo[1] + ((i >> 1) & 1) * half, lo[2] + ((i >> 2) & 1) * half};
            if (!overlaps(cl, half)) continue;
            uint64_t cp;
            if (svo) {
                cp = (uint64_t)w_[p] + 2ull * r;
                if (!in(cp, 2)) return;
            } else {
                if (!in(p + 1 + r, 1)) return;
                cp = w_[p + 1 + r];
                if (!in(cp, 1)) return;
            }
            if (depth + 1 == L.e[0]) emit(k, w_[cp], cl);
            else node(k, (uint32_t)cp, depth + 1, cl);
            if (err_) return;
        }
    }
    const Spec& sp_;
    const uint32_t* w_;
    uint64_t nw_;
    uint32_t* out_;
    int nlev_;
    int s_[kMaxFormatLevels];
    int64_t side_;
    int64_t c0_[3];
    int err_ = 0;
};

}  // namespace

VoxelSource* make_dense_source(const uint32_t* words, const int ldim[3]) {
    return new DenseSource(words, nullptr, nullptr, ldim);
}
VoxelSource* make_palette_source(const uint8_t* idx, const uint32_t* palette, const int ldim[3]) {
    return new DenseSource(nullptr, idx, palette, ldim);
}
VoxelSource* make_brick_source(const vx_grid* g) { return new BrickSource(g); }

int build_canonical(const Spec& spec, VoxelSource& src, int dedup_scope, BuildResult* out, int threads) {
    Builder b(spec, src, dedup_scope, *out);
    if (threads != 1 && src.thread_safe() && spec.lv.size() >= 2 &&
        (spec.lv[0].kind == K_RAW || spec.lv[0].kind == K_DF))
        return b.run_parallel(threads > 0 ? threads : omp_get_max_threads());
    return b.run();
}

int decode_cube(const Spec& spec, const uint32_t* words, uint64_t nwords, int64_t x0, int64_t y0, int64_t z0,
                int log2s, uint32_t* out) {
    const int64_t c0[3] = {x0, y0, z0};
    Decoder d(spec, words, nwords, c0, log2s, out);
    return d.run();
}

}  // namespace vx
