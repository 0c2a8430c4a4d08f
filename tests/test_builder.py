"""Host-side tests of the product library (no GPU): the C ABI exports, the
format parser, and the Morton-order builder checked against the oracle's
independent decoder of the paper's layout and against hand-derived buffers."""
import json
import os
import re

import numpy as np
import pytest

import oracle
import synth
import paper_2410_14128_b300 as vx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def build(spec, grid, **kw):
    return vx.Volume(spec, grid, upload=False, **kw)


# ---------------------------------------------------------------------------
# ABI
# ---------------------------------------------------------------------------
def header_functions():
    with open(os.path.join(ROOT, "include", "vx.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(vx_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_header_function():
    import ctypes
    names = header_functions()
    assert len(names) >= 12
    L = ctypes.CDLL(vx.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(vx.exported_symbols())
    assert vx.lib().vx_version() >= 10000


def test_binding_argument_counts_match_header():
    # every C declaration and its ctypes signature take the same number of
    # arguments (a parameter added on one side only would shift the rest)
    with open(os.path.join(ROOT, "include", "vx.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    decls = re.findall(r"^(?:int|const char\*)\s+(vx_\w+)\s*\(([^;]*?)\)\s*;", text, flags=re.M | re.S)
    assert {n for n, _ in decls} == set(header_functions())
    for name, params in decls:
        p = params.strip()
        count = 0 if p in ("", "void") else p.count(",") + 1
        assert len(vx._SIGS[name][1]) == count, name


def test_struct_layouts_match_header(tmp_path):
    # the ctypes mirrors of the C structs have the header's sizes and offsets
    import ctypes
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "vx.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(vx_stats), '
                   'offsetof(vx_stats, upload_ms), offsetof(vx_stats, tuned), offsetof(vx_stats, tuned_opts), '
                   'sizeof(vx_trace_opts), sizeof(vx_batch_item)); '
                   'printf("%zu %zu\\n", sizeof(vx_build_opts), offsetof(vx_build_opts, generic_kernel)); '
                   'return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(vx._Stats), vx._Stats.upload_ms.offset, vx._Stats.tuned.offset,
            vx._Stats.tuned_opts.offset, ctypes.sizeof(vx._TraceOpts), ctypes.sizeof(vx._BatchItem),
            ctypes.sizeof(vx._BuildOpts), vx._BuildOpts.generic_kernel.offset]
    assert got == want


def test_compiled_formats_are_the_instantiated_ones():
    # vx_formats lists every format composed at compile time, once, in the
    # spelling of its instantiation
    import glob
    text = "".join(open(f).read() for f in glob.glob(os.path.join(ROOT, "paper_2410_14128_b300", "csrc",
                                                                  "formats_*.cu")))
    listed = re.findall(r'^VX_FMT\(\w+, "([^"]+)"', text, flags=re.M)
    specs = vx.compiled_formats()
    assert len(specs) == len(set(specs)) == len(listed) >= 44
    assert sorted(specs) == sorted(listed)


def test_generic_kernel_option_selects_the_run_time_kernels():
    g = synth.value_noise_volume(101, 64)
    assert build("S(4) R(2,2,2)", g).stats()["specialized"]
    assert not build("S(4) R(2,2,2)", g, generic_kernel=True).stats()["specialized"]
    assert not build("S(2) R(4,4,4)", g).stats()["specialized"]  # not compiled in


def test_stats_report_no_tuning_before_autotune():
    g = synth.random_grid(5, (16, 16, 16), 0.2)
    assert build("R(2,2,2) S(2)", g).stats()["tuned"] is None


def test_footprint_bytes_counts_marked_sectors():
    torch = pytest.importorskip("torch")
    words = np.zeros(5, np.uint32)
    words[0] = 0b1011            # sectors 0, 1, 3
    words[3] = 1 << 31           # sector 127
    words[4] = 0xFFFFFFFF        # sectors 128..159
    t = torch.from_numpy(words.view(np.int32))
    assert vx.Volume.footprint_bytes(t) == 32 * (3 + 1 + 32)


# ---------------------------------------------------------------------------
# Spec parser
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec,code", [
    ("", vx.VX_EINVAL), ("Q(3)", vx.VX_EINVAL), ("R(1,1)", vx.VX_EINVAL), ("S(0)", vx.VX_EINVAL),
    ("R(2,2,2) R(1,2,1)", vx.VX_EINVAL),            # lower levels must be cubic (Sec. 5)
    ("R(2,2,2) S(1)", vx.VX_EINVAL),                # 8^3 spec on a 16^3 grid
    ("D(2,2,2) R(2,2,2)", vx.VX_EINVAL),            # D takes (W,H,D,M) (Table 1)
    ("D(2,2,2,70000) R(2,2,2)", vx.VX_EINVAL),      # distance cap beyond the supported 65535
    ("R(2,2,2) D(1,2,1,3)", vx.VX_EINVAL),          # lower DF levels must be cubic too (Sec. 5)
])
def test_bad_specs_rejected(spec, code):
    g = np.zeros((16, 16, 16), np.uint32)
    with pytest.raises(vx.VxError) as e:
        build(spec, g)
    assert e.value.code == code


def test_n_cubed_shorthand_matches_explicit():
    g = synth.random_grid(3, (16, 16, 16), 0.1)
    a = build("R(2^3) G(2)", g).canonical()
    b = build("R(2, 2, 2) G(2)", g).canonical()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# Canonical buffer: bit-exact against hand-derived examples of the layout
# ---------------------------------------------------------------------------
def _layout():
    with open(os.path.join(GOLDEN, "layout_examples.json")) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", _layout(), ids=lambda e: e["name"])
def test_builder_reproduces_hand_built_buffers(ex):
    nx, ny, nz = ex["dims"]
    g = np.zeros((nz, ny, nx), np.uint32)
    for x, y, z, c in ex["voxels"]:
        g[z, y, x] = c
    words = build(ex["spec"], g).canonical()
    exp = np.zeros(ex["nwords"], np.uint32)
    for k, v in ex["set"].items():
        exp[int(k)] = v
    assert words.tolist() == exp.tolist()


# ---------------------------------------------------------------------------
# decode(build(G)) == G for many formats, by the oracle's decoder
# ---------------------------------------------------------------------------
SPECS_16 = ["R(4,4,4)", "S(4)", "G(4)", "R(2,2,2) R(2,2,2)", "R(1,1,1) S(1) G(2)", "S(2) R(2,2,2)",
            "G(2) S(2)", "R(3,3,3) G(1)", "S(1) S(1) S(1) S(1)", "R(2,2,2) S(1) G(1)", "G(1) R(3,3,3)",
            "D(4,4,4,6)", "D(2,2,2,3) R(2,2,2)", "R(2,2,2) D(2,2,2,2)", "D(1,1,1,1) S(1) G(2)",
            "D(2,2,2,6) D(2,2,2,6)", "G(2) D(2,2,2,1)"]


@pytest.mark.parametrize("spec", SPECS_16)
@pytest.mark.parametrize("p", [0.0, 0.03, 0.3, 1.0])
def test_decode_roundtrip_oracle(spec, p):
    g = synth.random_grid(hash((spec, p)) & 0xFFFF, (16, 16, 16), p, colors=3)
    v = build(spec, g)
    words = v.canonical()
    assert np.array_equal(oracle.decode(words, spec), g)
    assert np.array_equal(v.decode_brick(0, 0, 0, 4), g)
    assert np.array_equal(v.decode_brick(8, 0, 8, 3), g[8:16, 0:8, 8:16])
    assert v.stats()["occupied_voxels"] == int((g != 0).sum())


@pytest.mark.parametrize("spec", ["R(1,0,2) R(2,2,2)", "R(3,1,2) S(2)", "R(0,2,1) G(2)"])
def test_non_cubic_top_level(spec):
    (lx, ly, lz), _ = oracle.spec_dims(spec)
    g = synth.random_grid(9, (1 << lz, 1 << ly, 1 << lx), 0.2)
    words = build(spec, g).canonical()
    assert np.array_equal(oracle.decode(words, spec), g)


def test_terrain_roundtrip_64():
    g = synth.terrain_volume(5, 64)
    for spec in ["R(2,2,2) S(2) G(2)", "R(2,2,2) R(2,2,2) R(2,2,2)", "S(4) R(2,2,2)", "G(6)"]:
        assert np.array_equal(oracle.decode(build(spec, g).canonical(), spec), g), spec


def test_brick_callback_matches_dense():
    g = synth.random_grid(21, (32, 32, 32), 0.05)

    def fill(user, x0, y0, z0, l2, out):
        s = 1 << l2
        blk = np.ascontiguousarray(g[z0:z0 + s, y0:y0 + s, x0:x0 + s]).reshape(-1)
        np.ctypeslib.as_array(out, shape=(s * s * s,))[:] = blk
        return 0

    for spec in ["R(2,2,2) G(3)", "S(3) R(2,2,2)"]:
        a = build(spec, g).canonical()
        b = vx.Volume(spec, log2_dim=(5, 5, 5), fill_brick=fill, upload=False).canonical()
        assert np.array_equal(a, b), spec


# ---------------------------------------------------------------------------
# Invariants and closed forms
# ---------------------------------------------------------------------------
def test_empty_volume_is_one_word():
    g = np.zeros((16, 16, 16), np.uint32)
    for spec in SPECS_16:
        w = build(spec, g).canonical()
        assert w.tolist() == [0], spec


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_full_grid_closed_forms(L):
    n = 1 << L
    g = np.full((n, n, n), 0xFF00FF00, np.uint32)
    s = build(f"S({L})", g).stats()
    nodes = sum(8 ** d for d in range(L + 1))  # every node of a complete octree, leaves included
    assert s["level_nodes"][0] == nodes
    assert s["canonical_words"] == 1 + 2 * nodes
    d = build(f"G({L})", g).stats()
    # one distinct node per depth: L internal nodes (8 pointers each) and one leaf word
    assert d["level_nodes"][0] == L + 1
    assert d["canonical_words"] == 1 + 1 + 9 * L
    r = build(f"R({L},{L},{L})", g).stats()
    assert r["canonical_words"] == 1 + n ** 3


@pytest.mark.parametrize("seed,p", [(1, 0.02), (2, 0.2), (3, 0.6)])
def test_svdag_never_larger_than_svo(seed, p):
    g = synth.random_grid(seed, (32, 32, 32), p, colors=2)
    for top in ["", "R(1,1,1) ", "R(2,2,2) "]:
        L = 5 - (0 if not top else int(top[2]))
        so = build(f"{top}S({L})", g).stats()
        dg = build(f"{top}G({L})", g).stats()
        k = 0 if not top else 1
        assert dg["level_nodes"][k] <= so["level_nodes"][k]


@pytest.mark.parametrize("spec", ["R(2,2,2) G(3)", "R(3,3,3) G(2)", "S(2) G(3)"])
def test_whole_level_dedup_never_larger(spec):
    g = synth.terrain_volume(8, 32)
    whole = build(spec, g, dedup=vx.DEDUP_WHOLE_LEVEL)
    per = build(spec, g, dedup=vx.DEDUP_PER_SUBVOLUME)
    assert whole.stats()["canonical_words"] <= per.stats()["canonical_words"]
    assert np.array_equal(oracle.decode(per.canonical(), spec), g)
    assert np.array_equal(oracle.decode(whole.canonical(), spec), g)


def test_single_colour_dedups_strongly():
    # a single-coloured volume shares sub-volume interiors across the level
    g = synth.random_grid(4, (32, 32, 32), 0.5, colors=1)
    g[:, :16, :] = np.uint32(0xFF0000FF)
    whole = build("R(2,2,2) G(3)", g, dedup=vx.DEDUP_WHOLE_LEVEL).stats()["canonical_words"]
    per = build("R(2,2,2) G(3)", g, dedup=vx.DEDUP_PER_SUBVOLUME).stats()["canonical_words"]
    assert whole < per


@pytest.mark.parametrize("spec", ["R(2,2,2) G(3)", "R(2,2,2) S(3)", "R(3,3,3) R(1,1,1) G(1)", "R(1,0,2) S(1) G(2)",
                                  "R(2,2,2) S(1) R(1,1,1) G(1)", "D(2,2,2,6) G(3)", "D(3,1,2,4) D(2,2,2,6) R(1,1,1)"])
@pytest.mark.parametrize("dedup", [vx.DEDUP_WHOLE_LEVEL, vx.DEDUP_PER_SUBVOLUME])
def test_parallel_build_equals_sequential(spec, dedup):
    (lx, ly, lz), _ = oracle.spec_dims(spec)
    g = synth.terrain_volume(33, 1 << max(lx, ly, lz))[: 1 << lz, : 1 << ly, : 1 << lx]
    g = np.ascontiguousarray(g)
    seq = build(spec, g, dedup=dedup, threads=1)
    par = build(spec, g, dedup=dedup, threads=0)
    assert np.array_equal(seq.canonical(), par.canonical())
    a, b = seq.stats(), par.stats()
    for key in ("canonical_words", "occupied_voxels", "level_words", "level_nodes"):
        assert a[key] == b[key], key
    assert np.array_equal(oracle.decode(par.canonical(), spec), g)


def test_parallel_build_palette_grid():
    g8 = np.random.default_rng(5).integers(0, 4, size=(64, 64, 64)).astype(np.uint8)
    g8[g8 == 3] = 0
    pal = np.zeros(256, np.uint32)
    pal[1:3] = [0xFF0000FF, 0xFF00FF00]
    seq = vx.Volume("R(2,2,2) G(4)", g8, palette=pal, upload=False, threads=1)
    par = vx.Volume("R(2,2,2) G(4)", g8, palette=pal, upload=False, threads=0)
    assert np.array_equal(seq.canonical(), par.canonical())
    assert np.array_equal(oracle.decode(par.canonical(), "R(2,2,2) G(4)"), pal[g8])


# ---------------------------------------------------------------------------
# DF levels: distances by the oracle's definition (checked inside decode),
# size, and the cap
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["D(5,5,5,6)", "D(3,3,3,6) R(2,2,2)", "D(2,2,2,2) D(3,3,3,6)", "R(1,1,1) D(2,2,2,9) G(2)"])
def test_df_distances_match_definition(spec):
    g = synth.terrain_volume(41, 32)
    v = build(spec, g)
    assert np.array_equal(oracle.decode(v.canonical(), spec), g)


def test_df_words_are_twice_raw():
    g = synth.random_grid(42, (32, 32, 32), 0.05)
    raw = build("R(3,3,3) R(2,2,2)", g).stats()
    df = build("D(3,3,3,6) R(2,2,2)", g).stats()
    assert df["level_words"][0] == 2 * raw["level_words"][0]
    assert df["level_words"][1] == raw["level_words"][1]
    assert df["canonical_words"] == raw["canonical_words"] + raw["level_words"][0]


def test_df_cap_closed_form():
    # one voxel at the origin of a 16^3 D level: every cell stores min(x + y + z, M)
    g = np.zeros((16, 16, 16), np.uint32)
    g[0, 0, 0] = 0xFF0000FF
    for M in (0, 1, 5, 45, 65535):
        w = build(f"D(4,4,4,{M})", g).canonical()
        d = w[1 + 1::2][: 16 ** 3].reshape(16, 16, 16)
        z, y, x = np.indices((16, 16, 16))
        assert np.array_equal(d, np.minimum(x + y + z, M)), M


# ---------------------------------------------------------------------------
# vx_load: word buffers validated against the layout, save / open round trip
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["R(2,2,2) S(1) G(1)", "D(2,2,2,3) R(2,2,2)", "S(2) G(2)", "G(4)", "R(1,1,1) S(1) G(2)"])
def test_load_validated_roundtrip(spec, tmp_path):
    g = synth.random_grid(51, (16, 16, 16), 0.15, colors=3)
    v = build(spec, g)
    w = v.canonical()
    u = vx.Volume.load(spec, w, upload=False)
    assert np.array_equal(u.canonical(), w)
    a, b = v.stats(), u.stats()
    assert a["canonical_words"] == b["canonical_words"]
    assert a["level_words"] == b["level_words"] and a["level_nodes"] == b["level_nodes"]
    assert np.array_equal(u.decode_brick(0, 0, 0, 4), g)
    v.save(str(tmp_path / "vol.npz"))
    r = vx.Volume.open(str(tmp_path / "vol.npz"), upload=False)
    assert r.spec == spec and np.array_equal(r.canonical(), w)


@pytest.mark.parametrize("ex", _layout(), ids=lambda e: e["name"])
def test_load_accepts_hand_built_buffers(ex):
    w = np.zeros(ex["nwords"], np.uint32)
    for k, val in ex["set"].items():
        w[int(k)] = val
    vx.Volume.load(ex["spec"], w, upload=False)


def _malformed():
    with open(os.path.join(GOLDEN, "layout_examples.json")) as f:
        return json.load(f)["malformed"]


@pytest.mark.parametrize("ex", _malformed(), ids=lambda e: e["name"])
def test_load_rejects_malformed_buffers(ex):
    w = np.zeros(ex["nwords"], np.uint32)
    for k, val in ex["set"].items():
        w[int(k)] = val
    with pytest.raises(vx.VxError) as e:
        vx.Volume.load(ex["spec"], w, upload=False)
    assert e.value.code == vx.VX_EINVAL
    vx.Volume.load(ex["spec"], w, upload=False, validate=False)  # the walk is skipped


def test_load_rejects_corruption_anywhere():
    g = synth.terrain_volume(52, 32)
    spec = "R(2,2,2) S(1) G(2)"
    w = build(spec, g).canonical()
    rng = np.random.default_rng(53)
    rejected = 0
    for _ in range(40):
        bad = w.copy()
        i = int(rng.integers(1, len(w)))
        bad[i] = np.uint32(len(w) + int(rng.integers(1, 1 << 20)))  # a pointer past the end, or a wrong word
        try:
            vx.Volume.load(spec, bad, upload=False)
        except vx.VxError:
            rejected += 1
    assert rejected >= 20  # most corruptions hit a pointer or a mask; RGBA words may take any value


def test_load_refuses_buffers_beyond_the_word_limit():
    # Sec. 3.3: 32-bit word offsets, so at most 2^32 - 1 words; the size is
    # checked before any word is read (the 4-word array stands for a huge one)
    import ctypes
    w = np.zeros(4, np.uint32)
    o = vx._BuildOpts(vx.DEDUP_WHOLE_LEVEL, -1, 1, 0, 0)
    h = ctypes.c_void_p()
    rc = vx.lib().vx_load(b"G(2)", ctypes.c_void_p(w.ctypes.data), 1 << 32, ctypes.byref(o), 1, ctypes.byref(h))
    assert rc == vx.VX_ETOOBIG and not h.value
    rc = vx.lib().vx_load(b"G(2)", ctypes.c_void_p(w.ctypes.data), 0, ctypes.byref(o), 1, ctypes.byref(h))
    assert rc == vx.VX_EINVAL and not h.value
