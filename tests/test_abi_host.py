"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point include/gsr.h declares, and validates arguments on the
host with a host-only context."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    from paper_2311_11700_gb300 import build
    build.build()
    import paper_2311_11700_gb300 as g
    g.lib()
    return g


def _declared():
    h = open(os.path.join(ROOT, "include", "gsr.h")).read()
    return sorted(set(re.findall(r"GS_API\s+[\w\s\*]+?\b(gs_\w+)\s*\(", h)))


def test_every_declared_symbol_is_exported_and_bound(G):
    names = _declared()
    assert len(names) >= 10
    L = ctypes.CDLL(G.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
        assert n in G.ABI, f"binding does not wrap {n}"


def test_struct_layouts_match_the_c_compiler(G, tmp_path):
    """The ctypes mirror has the sizes and field offsets gcc gives the header's structs."""
    import subprocess
    src = tmp_path / "layout.c"
    fields = {"gs_scene": [f for f, _ in G.gs_scene._fields_], "gs_view": [f for f, _ in G.gs_view._fields_],
              "gs_images": [f for f, _ in G.gs_images._fields_], "gs_grads": [f for f, _ in G.gs_grads._fields_],
              "gs_layout": [f for f, _ in G.gs_layout._fields_],
              **{st: [f for f, _ in getattr(G, st)._fields_] for st in ("gs_expand_params", "gs_scene_out",
                                                                         "gs_densify_params", "gs_tune_result",
                                                                         "gs_timing")}}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gsr.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for st, fs in fields.items():
        cls = getattr(G, st)
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fs:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, f"{st}.{f}"


class _FakeScene:
    """Stands in for Scene with fake device pointers: queries never dereference."""

    def __init__(self, n, deg=0, null=False):
        self.n, self.sh_degree, self.null = n, deg, null

    def c_struct(self):
        import paper_2311_11700_gb300 as g
        p = None if self.null else 0x1000
        return g.gs_scene(self.n, self.sh_degree, 0, p, p, p, p, p, None)


def _view(W=160, H=120, scene=0):
    return dict(width=W, height=H, fx=120.0, fy=120.0, cx=W / 2, cy=H / 2, z_near=0.2, bg=(0, 0, 0),
                T_cw=np.concatenate([np.eye(3), np.zeros((3, 1))], 1).reshape(12), scene=scene)


@pytest.fixture(scope="module")
def hctx(G):
    return G.Context(-1)


def test_host_only_context_answers_queries(G, hctx):
    n1 = G.gs_workspace_query(hctx, [_FakeScene(2000)], [_view()], 10_000)
    n2 = G.gs_workspace_query(hctx, [_FakeScene(2000)], [_view()], 20_000)
    assert abs((n2 - n1) - 8 * 10_000) <= 512  # two u32 pair arrays (lists, large-sort scratch)
    lay = G.gs_workspace_layout(hctx, [_FakeScene(300), _FakeScene(1000)], [_view(), _view(64, 48, 1)], 4096)
    assert lay.n_splats == 512 + 1024
    assert list(lay.splat_off[:2]) == [0, 512]
    assert lay.n_tiles == 10 * 8 + 4 * 3
    assert list(lay.tile_off[:2]) == [0, 80]
    for f in ("rec", "rect", "ntiles", "dkey", "ranges", "pair_val"):
        assert getattr(lay, f) % 256 == 0


@pytest.mark.parametrize("case", ["n_views0", "deg4", "size0", "scene_idx", "pairs0", "null_plane", "fx0",
                                  "too_many_views"])
def test_host_validation(G, hctx, case):
    sc, vw, mp = [_FakeScene(100)], [_view()], 1000
    if case == "n_views0":
        vw = []
    elif case == "deg4":
        sc = [_FakeScene(100, 4)]
    elif case == "size0":
        vw = [_view(0, 10)]
    elif case == "scene_idx":
        vw = [_view(scene=3)]
    elif case == "pairs0":
        mp = 0
    elif case == "null_plane":
        sc = [_FakeScene(100, null=True)]
    elif case == "fx0":
        v = _view()
        v["fx"] = 0.0
        vw = [v]
    elif case == "too_many_views":
        vw = [_view()] * 33
    if not vw:
        # an empty array still needs a valid pointer for ctypes
        arr_s = (G.gs_scene * 1)(sc[0].c_struct())
        arr_v = (G.gs_view * 1)()
        n = ctypes.c_size_t()
        st = G.lib().gs_workspace_query(hctx.handle, arr_s, 1, arr_v, 0, mp, ctypes.byref(n))
        assert st == G.GS_ERR_INVALID_ARG
        return
    with pytest.raises(G.GsrError) as e:
        G.gs_workspace_query(hctx, sc, vw, mp)
    assert e.value.status == G.GS_ERR_INVALID_ARG


def test_timing_modes(G, hctx):
    # 0 off, 1 events + work counters, 2 events only; anything else is refused
    for on in (0, 1, 2, 0):
        G.gs_ctx_set_timing(hctx, on)
    for bad in (-1, 3):
        with pytest.raises(G.GsrError) as e:
            G.gs_ctx_set_timing(hctx, bad)
        assert e.value.status == G.GS_ERR_INVALID_ARG


def test_host_only_context_refuses_launches(G, hctx):
    arr_s = (G.gs_scene * 1)(_FakeScene(10).c_struct())
    arr_v = (G.gs_view * 1)(G.view_struct(_view()))
    img = G.gs_images(None, None, None)
    need = G.gs_workspace_query(hctx, [_FakeScene(10)], [_view()], 100)
    st = G.lib().gs_render_forward(hctx.handle, arr_s, 1, arr_v, 1, ctypes.c_void_p(0x100000), need, 100,
                                   ctypes.byref(img), None)
    assert st == G.GS_ERR_UNSUPPORTED


def test_autotune_cache_text_round_trip(G, hctx, tmp_path):
    src = tmp_path / "in.txt"
    src.write_text("# header\nv640x480:0;s19:3; 16 16 1 0 0 0.25 0.5\nv320x240:0;s17:0; 8 8 0 0 1 0.1 0.2\n")
    ctx = G.Context(-1)
    ctx.autotune_load(src)
    out = tmp_path / "out.txt"
    ctx.autotune_save(out)
    lines = sorted(l for l in out.read_text().splitlines() if not l.startswith("#"))
    assert lines == sorted(["v640x480:0;s19:3; 16 16 1 0 0 0.25 0.5", "v320x240:0;s17:0; 8 8 0 0 1 0.1 0.2"])


@pytest.mark.parametrize("line", ["v1x1:0; 16 16 1 0", "v1x1:0; 7 7 0 0 0 1 1", "v1x1:0; 16 16 9 0 0 1 1",
                                  "v1x1:0; 16 16 0 0 2 1 1"])
def test_autotune_cache_rejects_bad_lines(G, hctx, tmp_path, line):
    src = tmp_path / "bad.txt"
    src.write_text(line + "\n")
    with pytest.raises(G.GsrError) as e:
        G.Context(-1).autotune_load(src)
    assert e.value.status == G.GS_ERR_INVALID_ARG


def test_step_autotune_host_checks(G, hctx, tmp_path):
    """gs_autotune_step_l1 validates its arguments and reps on the host, refuses a
    host-only context, and its cache keys (parameter step "step:", pose-only step
    "pose:") survive the text round trip beside the separate-call keys."""
    arr_s = (G.gs_scene * 1)(_FakeScene(10).c_struct())
    arr_v = (G.gs_view * 1)(G.view_struct(_view()))
    img = G.gs_images(None, None, None)
    need = G.gs_workspace_query(hctx, [_FakeScene(10)], [_view()], 100)
    ws, loss, tw, tgt = (ctypes.c_void_p(a) for a in (0x100000, 0x200000, 0x300000, 0x400000))
    res = G.gs_tune_result()

    def call(loss_p=loss, tw_p=tw, reps=1, result=True):
        return G.lib().gs_autotune_step_l1(hctx.handle, arr_s, 1, arr_v, 1, ws, need, 100, ctypes.byref(img), tgt,
                                           tgt, 1.0, 0.5, loss_p, None, tw_p, 0, reps, 0,
                                           ctypes.byref(res) if result else None, None)

    assert call(result=False) == G.GS_ERR_INVALID_ARG
    assert call(loss_p=None) == G.GS_ERR_INVALID_ARG
    assert call(tw_p=None) == G.GS_ERR_INVALID_ARG  # neither parameter gradients nor the twist
    assert call(reps=0) == G.GS_ERR_INVALID_ARG
    assert call(reps=101) == G.GS_ERR_INVALID_ARG
    assert call() == G.GS_ERR_UNSUPPORTED
    src = tmp_path / "in.txt"
    keys = ["step:v640x480:0;s19:3; 16 16 2 2 0 0.25 0", "pose:v640x480:0;s19:3; 16 8 0 0 1 0.5 0",
            "v640x480:0;s19:3; 16 16 2 3 0 0.1 0.2"]
    src.write_text("\n".join(keys) + "\n")
    ctx = G.Context(-1)
    ctx.autotune_load(src)
    out = tmp_path / "out.txt"
    ctx.autotune_save(out)
    assert sorted(l for l in out.read_text().splitlines() if not l.startswith("#")) == sorted(keys)
