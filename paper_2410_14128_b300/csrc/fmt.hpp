// fmt.hpp -- description of a hybrid format as a stack of "node levels",
// shared by the host code and the CUDA kernels.
//
// A format is a list of the paper's base formats (Sec. 3.1, Table 1).  For
// traversal every level is expanded into node levels: a Raw level R(W,H,D)
// or a DF level D(W,H,D,M) is one node level with 2^W x 2^H x 2^D children
// (a DF cell also stores its L1 distance to the nearest non-empty cell, which
// the traversal uses to skip look-ups); an SVO or SVDAG level of
// depth L is L node levels with 2 x 2 x 2 children each (the octree nodes of
// Sec. 3.3).  Node level j's children are cubes of side 2^s_j voxels; all
// levels but the first are cubic (Sec. 5), so s_j is one number per level.
//
// Everything a kernel needs about the format is packed into a few integers,
// so that a compile-time format (template argument) and a run-time format
// (kernel argument) run the same code.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define VX_HD __host__ __device__
#else
#define VX_HD
#endif

namespace vx {

enum Kind : int { K_RAW = 0, K_SVO = 1, K_DAG = 2, K_DF = 3 };

constexpr int kMaxFormatLevels = 16;
constexpr int kMaxNodeLevels = 16;
constexpr int kMaxLog2Dim = 15;

struct FmtParams {
    uint32_t J;        // node levels
    uint32_t kind;     // 2 bits per node level (Kind)
    uint32_t top;      // bit j: node level j is the root of its format level
    uint32_t bot;      // bit j: node level j's children are terminating integers
    uint64_t s;        // 4 bits per node level: log2 side of its children
    uint64_t b;        // 4 bits per node level: log2 children per axis (levels >= 1)
    uint32_t b0[3];    // node level 0: log2 children per axis
    uint32_t ldim[3];  // log2 grid side per axis
    uint64_t jpop;     // 4 bits per voxel bit h: deepest node level whose node spans bit h
};

struct LevelDesc {
    int kind;
    int e[3];  // Raw / DF: W,H,D;  SVO/SVDAG: L,L,L
};

// Expands format levels into node levels.  Returns false when the format
// cannot be expressed (too many levels, non-cubic lower level, bad extents).
constexpr bool make_fmt_params(const LevelDesc* lv, int n, FmtParams* out) {
    FmtParams p{};
    if (n < 1 || n > kMaxFormatLevels) return false;
    int kind[kMaxNodeLevels] = {};
    int bx[kMaxNodeLevels] = {}, by[kMaxNodeLevels] = {}, bz[kMaxNodeLevels] = {};
    int J = 0;
    uint32_t top = 0, bot = 0;
    for (int k = 0; k < n; k++) {
        const LevelDesc& L = lv[k];
        if (L.kind == K_RAW || L.kind == K_DF) {
            if (L.e[0] < 0 || L.e[1] < 0 || L.e[2] < 0) return false;
            if (L.e[0] + L.e[1] + L.e[2] == 0) return false;
            if (k > 0 && (L.e[0] != L.e[1] || L.e[1] != L.e[2])) return false;
            if (J >= kMaxNodeLevels) return false;
            kind[J] = L.kind; bx[J] = L.e[0]; by[J] = L.e[1]; bz[J] = L.e[2];
            top |= 1u << J; bot |= 1u << J;
            J++;
        } else if (L.kind == K_SVO || L.kind == K_DAG) {
            if (L.e[0] < 1) return false;
            for (int d = 0; d < L.e[0]; d++) {
                if (J >= kMaxNodeLevels) return false;
                kind[J] = L.kind; bx[J] = by[J] = bz[J] = 1;
                if (d == 0) top |= 1u << J;
                if (d == L.e[0] - 1) bot |= 1u << J;
                J++;
            }
        } else {
            return false;
        }
    }
    int ld[3] = {0, 0, 0};
    for (int j = 0; j < J; j++) { ld[0] += bx[j]; ld[1] += by[j]; ld[2] += bz[j]; }
    for (int i = 0; i < 3; i++)
        if (ld[i] > kMaxLog2Dim) return false;
    // s_j: side of node level j's children = sum of deeper levels' fanouts
    // (the same on every axis, since deeper levels are cubic).
    int s[kMaxNodeLevels + 1] = {};
    s[J] = 0;
    for (int j = J - 1; j >= 0; j--) s[j] = (j + 1 < J ? s[j + 1] + bx[j + 1] : 0);
    p.J = (uint32_t)J;
    for (int j = 0; j < J; j++) {
        p.kind |= (uint32_t)kind[j] << (2 * j);
        p.s |= (uint64_t)s[j] << (4 * j);
        if (j > 0) {
            if (bx[j] > 15) return false;
            p.b |= (uint64_t)bx[j] << (4 * j);
        }
    }
    p.top = top;
    p.bot = bot;
    p.b0[0] = (uint32_t)bx[0]; p.b0[1] = (uint32_t)by[0]; p.b0[2] = (uint32_t)bz[0];
    p.ldim[0] = (uint32_t)ld[0]; p.ldim[1] = (uint32_t)ld[1]; p.ldim[2] = (uint32_t)ld[2];
    // jpop[h]: the deepest node level j >= 1 whose node spans 2^s_{j-1} > 2^h
    // voxels, i.e. the level to resume at after a step that changes voxel
    // coordinate bit h; 0 if none (the root node spans the whole grid).
    for (int h = 0; h < 16; h++) {
        int best = 0;
        for (int j = 1; j < J; j++)
            if (s[j - 1] > h) best = j;
        p.jpop |= (uint64_t)best << (4 * h);
    }
    *out = p;
    return true;
}

VX_HD inline int fp_kind(const FmtParams& p, int j) { return (int)((p.kind >> (2 * j)) & 3u); }
VX_HD inline int fp_s(const FmtParams& p, int j) { return (int)((p.s >> (4 * j)) & 15u); }
VX_HD inline int fp_b(const FmtParams& p, int j) { return (int)((p.b >> (4 * j)) & 15u); }
VX_HD inline int fp_jpop(const FmtParams& p, int h) { return (int)((p.jpop >> (4 * h)) & 15u); }

}  // namespace vx
