// spec.cpp -- format signatures (Table 1: R(W,H,D), S(L), G(L); extents are
// log2 per axis, so R(1,0,2) is a 2x1x4 grid, Sec. 3.2), error reporting and
// Morton-order helpers (Sec. 5, Fig. 5).
#include <stdarg.h>
#include <stdio.h>

#include <cctype>
#include <string>

#include "vx_internal.hpp"

namespace vx {

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

}  // namespace vx

extern "C" const char* vx_last_error(void) { return vx::g_err.c_str(); }

extern "C" int vx_version(void) { return 10000; }

namespace vx {

int parse_spec(const char* text, Spec* out) {
    if (!text) return fail(VX_EINVAL, "format spec is NULL");
    Spec sp;
    const char* s = text;
    auto skip = [&]() {
        while (*s == ' ' || *s == '\t' || *s == '\n') s++;
    };
    while (true) {
        skip();
        if (*s == ',') { s++; continue; }
        if (!*s) break;
        char k = (char)toupper((unsigned char)*s++);
        if (k != 'R' && k != 'S' && k != 'G' && k != 'D')
            return fail(VX_EINVAL, "spec '%s': unknown level kind '%c'", text, k);
        skip();
        if (*s++ != '(') return fail(VX_EINVAL, "spec '%s': expected '(' after %c", text, k);
        int vals[4], nv = 0;
        while (true) {
            skip();
            if (!isdigit((unsigned char)*s)) return fail(VX_EINVAL, "spec '%s': expected a number", text);
            long x = 0;
            while (isdigit((unsigned char)*s)) {
                x = 10 * x + (*s++ - '0');
                if (x > kMaxDfCap) return fail(VX_EINVAL, "spec '%s': number too large", text);
            }
            skip();
            if (*s == '^') {
                s++;
                skip();
                if (*s++ != '3' || nv + 3 > 4) return fail(VX_EINVAL, "spec '%s': only N^3 is allowed", text);
                vals[nv++] = (int)x; vals[nv++] = (int)x; vals[nv++] = (int)x;
            } else {
                if (nv >= 4) return fail(VX_EINVAL, "spec '%s': too many arguments", text);
                vals[nv++] = (int)x;
            }
            skip();
            if (*s == ',') { s++; continue; }
            if (*s == ')') { s++; break; }
            return fail(VX_EINVAL, "spec '%s': expected ',' or ')'", text);
        }
        Level L{};
        if (k == 'R') {
            if (nv != 3) return fail(VX_EINVAL, "spec '%s': R takes (W,H,D)", text);
            L.kind = K_RAW;
            L.e[0] = vals[0]; L.e[1] = vals[1]; L.e[2] = vals[2];
            if (L.e[0] + L.e[1] + L.e[2] == 0) return fail(VX_EINVAL, "spec '%s': R(0,0,0) holds one cell", text);
        } else if (k == 'D') {
            if (nv != 4) return fail(VX_EINVAL, "spec '%s': D takes (W,H,D,M)", text);
            L.kind = K_DF;
            L.e[0] = vals[0]; L.e[1] = vals[1]; L.e[2] = vals[2];
            L.m = vals[3];
            if (L.e[0] + L.e[1] + L.e[2] == 0) return fail(VX_EINVAL, "spec '%s': D(0,0,0,M) holds one cell", text);
        } else {
            if (nv != 1 || vals[0] < 1) return fail(VX_EINVAL, "spec '%s': %c takes one depth >= 1", text, k);
            L.kind = (k == 'S') ? K_SVO : K_DAG;
            L.e[0] = L.e[1] = L.e[2] = vals[0];
        }
        sp.lv.push_back(L);
    }
    if (sp.lv.empty()) return fail(VX_EINVAL, "spec '%s' has no levels", text);
    if ((int)sp.lv.size() > kMaxFormatLevels) return fail(VX_EINVAL, "spec '%s': too many levels", text);
    for (size_t k = 1; k < sp.lv.size(); k++) {
        const Level& L = sp.lv[k];
        if (L.e[0] != L.e[1] || L.e[1] != L.e[2])
            return fail(VX_EINVAL, "spec '%s': level %zu must be cubic (Morton construction, Sec. 5)", text, k + 1);
    }
    std::string c;
    for (size_t k = 0; k < sp.lv.size(); k++) {
        const Level& L = sp.lv[k];
        char buf[64];
        if (L.kind == K_RAW) snprintf(buf, sizeof buf, "R(%d,%d,%d)", L.e[0], L.e[1], L.e[2]);
        else if (L.kind == K_DF) snprintf(buf, sizeof buf, "D(%d,%d,%d,%d)", L.e[0], L.e[1], L.e[2], L.m);
        else snprintf(buf, sizeof buf, "%c(%d)", L.kind == K_SVO ? 'S' : 'G', L.e[0]);
        if (k) c += ' ';
        c += buf;
        for (int i = 0; i < 3; i++) sp.ldim[i] += L.e[i];
    }
    for (int i = 0; i < 3; i++)
        if (sp.ldim[i] > kMaxLog2Dim) return fail(VX_EINVAL, "spec '%s': grid side 2^%d too large", text, sp.ldim[i]);
    std::vector<LevelDesc> ld;
    for (const Level& L : sp.lv) ld.push_back(LevelDesc{L.kind, {L.e[0], L.e[1], L.e[2]}});
    if (!make_fmt_params(ld.data(), (int)ld.size(), &sp.fmt))
        return fail(VX_EINVAL, "spec '%s': more than %d octree/grid levels", text, kMaxNodeLevels);
    sp.canonical = c;
    *out = sp;
    return VX_OK;
}

void morton_decode(uint64_t m, const int e[3], uint32_t c[3]) {
    c[0] = c[1] = c[2] = 0;
    int bit = 0;
    for (int b = 0; b < 32; b++) {
        bool any = false;
        for (int i = 0; i < 3; i++) {
            if (b < e[i]) {
                c[i] |= (uint32_t)((m >> bit) & 1u) << b;
                bit++;
                any = true;
            }
        }
        if (!any) break;
    }
}

uint64_t morton_encode(const uint32_t c[3], const int e[3]) {
    uint64_t m = 0;
    int bit = 0;
    for (int b = 0; b < 32; b++) {
        bool any = false;
        for (int i = 0; i < 3; i++) {
            if (b < e[i]) {
                m |= (uint64_t)((c[i] >> b) & 1u) << bit;
                bit++;
                any = true;
            }
        }
        if (!any) break;
    }
    return m;
}

}  // namespace vx
