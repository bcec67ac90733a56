"""C ABI checks that need no GPU: the library loads, exports every function
include/retina.h declares, and its host-side validation rejects bad arguments
before anything is launched (RETINA_EINVAL / RETINA_ENOSPACE)."""
import ctypes

import pytest

from paper_1709_08610_gb300 import build as rbuild

rbuild.build()
from paper_1709_08610_gb300 import retina as rt  # noqa: E402

EINVAL, ENOSPACE = 1, 3
L = rt.lib
BOGUS = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails validation first
WS = ctypes.c_void_p(0x2000)  # a 256-byte-aligned bogus workspace, equally never dereferenced


def test_exports_every_declared_function():
    names = rt.header_functions()
    assert len(names) >= 11
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_and_version():
    assert L.retina_abi_version() == 2
    for c in range(5):
        assert L.retina_strerror(c)
    assert b"invalid" in L.retina_strerror(EINVAL)


def test_options_roundtrip_and_validation():
    old = rt.get_option(rt.OPT_LS_SEEDS_PER_WARP)
    rt.set_option(rt.OPT_LS_SEEDS_PER_WARP, 2)
    assert rt.get_option(rt.OPT_LS_SEEDS_PER_WARP) == 2
    rt.set_option(rt.OPT_LS_SEEDS_PER_WARP, old)
    assert L.retina_set_option(rt.OPT_LS_SEEDS_PER_WARP, 3) == EINVAL
    assert L.retina_set_option(rt.OPT_LS_SMEM_HITS, -1) == EINVAL
    assert L.retina_set_option(999, 1) == EINVAL
    rt.set_option(rt.OPT_BATCH_CTAS, 152)
    assert rt.get_option(rt.OPT_BATCH_CTAS) == 152
    rt.set_option(rt.OPT_BATCH_CTAS, 0)
    assert L.retina_set_option(rt.OPT_BATCH_CTAS, -1) == EINVAL
    for o in (rt.OPT_GRID_TC, rt.OPT_SEEDNET_TC):
        assert rt.get_option(o) == 1  # defaults
        rt.set_option(o, 0)
        assert rt.get_option(o) == 0
        rt.set_option(o, 1)
        assert L.retina_set_option(o, 2) == EINVAL


def _grid(lo=(-0.5, -0.5), step=(2 ** -10, 2 ** -10), n=(1024, 1024)):
    return rt.Grid(lo, step, n).c()


def test_workspace_size():
    b = ctypes.c_size_t()
    g = _grid()
    assert L.retina_grid_scan_workspace_size(1, 1, ctypes.byref(g), 0, 0, ctypes.byref(b)) == 0
    assert b.value >= 1024 * 1024 * 4  # the response grid lives in the workspace when not stored
    b2 = ctypes.c_size_t()
    assert L.retina_grid_scan_workspace_size(1, 1, ctypes.byref(g), 0, 1, ctypes.byref(b2)) == 0
    assert b2.value < b.value
    bad = _grid(step=(0.0, 1.0))
    assert L.retina_grid_scan_workspace_size(1, 1, ctypes.byref(bad), 0, 0, ctypes.byref(b)) == EINVAL
    # separable contraction is defined for the slope model only
    assert L.retina_grid_scan_workspace_size(1, 0, ctypes.byref(g), 2, 0, ctypes.byref(b)) == EINVAL


@pytest.mark.parametrize("sigma,K,model,flags", [(0.0, 8, 1, 0), (-1.0, 8, 1, 0), (float("nan"), 8, 1, 0),
                                                 (float("inf"), 8, 1, 0), (0.3, 0, 1, 0), (0.3, 8, 7, 0),
                                                 (0.3, 8, 0, 2), (0.3, 8, 1, 9)])
def test_grid_scan_rejects(sigma, K, model, flags):
    g = _grid()
    rc = L.retina_grid_scan(BOGUS, 10, BOGUS, None, 1, model, ctypes.byref(g), sigma, 1.0, flags, None, BOGUS, BOGUS,
                            BOGUS, BOGUS, K, BOGUS, 1 << 40, None)
    assert rc == EINVAL


def test_grid_scan_rejects_misaligned_and_small_workspace():
    g = _grid()
    rc = L.retina_grid_scan(ctypes.c_void_p(0x1004), 10, BOGUS, None, 1, 1, ctypes.byref(g), 0.3, 1.0, 0, None, BOGUS,
                            BOGUS, BOGUS, BOGUS, 8, BOGUS, 1 << 40, None)
    assert rc == EINVAL
    rc = L.retina_grid_scan(BOGUS, 10, BOGUS, None, 1, 1, ctypes.byref(g), 0.3, 1.0, 0, None, BOGUS, BOGUS, BOGUS, BOGUS,
                            8, BOGUS, 16, None)
    assert rc == ENOSPACE
    rc = L.retina_grid_scan(BOGUS, 10, None, None, 1, 1, ctypes.byref(g), 0.3, 1.0, 0, None, BOGUS, BOGUS, BOGUS, BOGUS,
                            8, BOGUS, 1 << 40, None)
    assert rc == EINVAL


def _opts(**kw):
    o = rt.LsOpts(**kw).c()
    return o


@pytest.mark.parametrize("mut", ["q0", "q9", "sigma0", "sigmanan", "c1neg", "c1one", "halv", "cap0", "upd-1", "upd3"])
def test_local_search_rejects(mut):
    o = _opts()
    if mut == "q0":
        o.q = 0
    elif mut == "q9":
        o.q = 9
    elif mut == "sigma0":
        o.sigma[1] = 0.0
    elif mut == "sigmanan":
        o.sigma[2] = float("nan")
    elif mut == "c1neg":
        o.c1 = -0.1
    elif mut == "c1one":
        o.c1 = 1.0
    elif mut == "halv":
        o.max_halvings = 31
    elif mut == "cap0":
        o.step_cap_cells = 0.0
    elif mut == "upd-1":
        o.update = -1
    elif mut == "upd3":
        o.update = 3
    g = _grid()
    rc = L.retina_local_search(BOGUS, 10, BOGUS, None, 1, 1, BOGUS, 16, ctypes.byref(o), ctypes.byref(g), BOGUS, BOGUS,
                               BOGUS, None, None)
    assert rc == EINVAL


def test_local_search_rejects_null_outputs_and_empty_is_ok():
    o = _opts()
    g = _grid()
    assert L.retina_local_search(BOGUS, 10, BOGUS, None, 1, 1, BOGUS, 16, ctypes.byref(o), ctypes.byref(g), None, BOGUS,
                                 BOGUS, None, None) == EINVAL
    # zero events or zero seeds: nothing to do, nothing launched
    assert L.retina_local_search(None, 0, None, None, 0, 1, None, 16, ctypes.byref(o), ctypes.byref(g), None, None, None,
                                 None, None) == 0
    assert L.retina_local_search(BOGUS, 10, BOGUS, None, 1, 1, BOGUS, 0, ctypes.byref(o), ctypes.byref(g), None, None,
                                 None, None, None) == 0


@pytest.mark.parametrize("mut", ["q0", "sigmanan", "c1one", "cap0", "K", "events", "model", "misaligned"])
def test_refine_maxima_rejects(mut):
    o = _opts()
    g = _grid()
    args = dict(hits=BOGUS, n_hits=10, E=1, model=1, K=16)
    if mut == "q0":
        o.q = 0
    elif mut == "sigmanan":
        o.sigma[0] = float("nan")
    elif mut == "c1one":
        o.c1 = 1.0
    elif mut == "cap0":
        o.step_cap_cells = 0.0
    elif mut == "K":
        args["K"] = -1
    elif mut == "events":
        args["E"] = 65536
    elif mut == "model":
        args["model"] = 7
    elif mut == "misaligned":
        args["hits"] = ctypes.c_void_p(0x1004)
    rc = L.retina_refine_maxima(args["hits"], args["n_hits"], BOGUS, None, args["E"], args["model"], BOGUS, BOGUS,
                                args["K"], ctypes.byref(o), ctypes.byref(g), BOGUS, BOGUS, BOGUS, WS, 1 << 20, None)
    assert rc == EINVAL


def test_refine_maxima_rejects_null_pointers_and_empty_is_ok():
    o = _opts()
    g = _grid()
    for k in range(6):
        ptrs = [BOGUS] * 5 + [WS]
        ptrs[k] = None  # theta_c, n_max, theta_out, R_out, status, workspace
        assert L.retina_refine_maxima(BOGUS, 10, BOGUS, None, 1, 1, ptrs[0], ptrs[1], 16, ctypes.byref(o),
                                      ctypes.byref(g), ptrs[2], ptrs[3], ptrs[4], ptrs[5], 1 << 20, None) == EINVAL
    assert L.retina_refine_maxima(BOGUS, 10, BOGUS, None, 1, 1, BOGUS, BOGUS, 16, None, ctypes.byref(g), BOGUS,
                                  BOGUS, BOGUS, WS, 1 << 20, None) == EINVAL
    # misaligned or short workspace
    assert L.retina_refine_maxima(BOGUS, 10, BOGUS, None, 1, 1, BOGUS, BOGUS, 16, ctypes.byref(o), ctypes.byref(g),
                                  BOGUS, BOGUS, BOGUS, ctypes.c_void_p(0x2010), 1 << 20, None) == EINVAL
    need = ctypes.c_size_t(0)
    assert L.retina_refine_maxima_workspace_size(3, ctypes.byref(need)) == 0 and need.value >= 5 * 4
    assert L.retina_refine_maxima(BOGUS, 10, BOGUS, None, 3, 1, BOGUS, BOGUS, 16, ctypes.byref(o), ctypes.byref(g),
                                  BOGUS, BOGUS, BOGUS, WS, need.value - 1, None) == ENOSPACE
    assert L.retina_refine_maxima_workspace_size(-1, ctypes.byref(need)) == EINVAL
    # zero events or K = 0: nothing to do, nothing launched
    assert L.retina_refine_maxima(None, 0, None, None, 0, 1, None, None, 16, ctypes.byref(o), ctypes.byref(g), None,
                                  None, None, None, 0, None) == 0
    assert L.retina_refine_maxima(BOGUS, 10, BOGUS, None, 1, 1, None, None, 0, ctypes.byref(o), ctypes.byref(g), None,
                                  None, None, None, 0, None) == 0


@pytest.mark.parametrize("mut", ["q0", "sigmanan", "c1one", "halv", "scale0", "capneg", "zrefinf", "events"])
def test_local_search4_rejects(mut):
    o = rt.LsOpts4().c()
    E = 1
    if mut == "q0":
        o.q = 0
    elif mut == "sigmanan":
        o.sigma[0] = float("nan")
    elif mut == "c1one":
        o.c1 = 1.0
    elif mut == "halv":
        o.max_halvings = 31
    elif mut == "scale0":
        o.scale[2] = 0.0
    elif mut == "capneg":
        o.step_cap = -1.0
    elif mut == "zrefinf":
        o.zref = float("inf")
    elif mut == "events":
        E = 65536
    assert L.retina_local_search4(BOGUS, 10, BOGUS, E, BOGUS, 16, None, ctypes.byref(o), BOGUS, BOGUS, BOGUS,
                                  None) == EINVAL


def test_local_search4_null_outputs_and_empty():
    o = rt.LsOpts4().c()
    assert L.retina_local_search4(BOGUS, 10, BOGUS, 1, BOGUS, 16, None, ctypes.byref(o), None, BOGUS, BOGUS,
                                  None) == EINVAL
    assert L.retina_local_search4(BOGUS, 10, BOGUS, 1, BOGUS, 16, None, None, BOGUS, BOGUS, BOGUS, None) == EINVAL
    assert L.retina_local_search4(None, 0, None, 0, None, 16, None, ctypes.byref(o), None, None, None, None) == 0
    assert L.retina_local_search4(BOGUS, 10, BOGUS, 1, None, 0, None, ctypes.byref(o), None, None, None, None) == 0


def test_pair_seeds4_and_extract4_reject_bad_arguments():
    lz = (ctypes.c_float * 2)(500.0, 700.0)
    ok = dict(dz=0.5, dmax=0.3, zlo=-250.0, zhi=250.0, zref=225.0)

    def ps(n_pairs=1, K=16, E=1, layer=lz, **kw):
        a = dict(ok, **kw)
        return L.retina_pair_seeds4(BOGUS, 10, BOGUS, E, layer, n_pairs, a["dz"], a["dmax"], a["zlo"], a["zhi"],
                                    a["zref"], BOGUS, BOGUS, K, None)
    assert ps(n_pairs=0) == EINVAL and ps(n_pairs=9) == EINVAL and ps(K=0) == EINVAL and ps(E=-1) == EINVAL
    assert ps(dmax=-1.0) == EINVAL and ps(dz=float("nan")) == EINVAL and ps(zhi=float("inf")) == EINVAL
    assert ps(layer=None) == EINVAL and ps(layer=(ctypes.c_float * 2)(float("nan"), 1.0)) == EINVAL
    assert L.retina_pair_seeds4(BOGUS, 10, None, 1, lz, 1, 0.5, 0.3, -1.0, 1.0, 0.0, BOGUS, BOGUS, 16, None) == EINVAL
    assert L.retina_pair_seeds4(None, 0, None, 0, lz, 1, 0.5, 0.3, -1.0, 1.0, 0.0, None, None, 16, None) == 0
    g = rt.Grid((-0.5, -0.5), (2 ** -10, 2 ** -10), (1024, 1024)).c()
    u = (ctypes.c_float * 4)(0.25, 0.25, 2 ** -10, 2 ** -10)
    bad_u = (ctypes.c_float * 4)(0.25, 0.0, 2 ** -10, 2 ** -10)

    def ex(n_points=100, K=8, units=u, merge=2.0, grid=g):
        return L.retina_extract_tracks4(BOGUS, BOGUS, None, None, 1, n_points, ctypes.byref(grid) if grid else None,
                                        units, 5.0, merge, BOGUS, BOGUS, None, BOGUS, K, None)
    assert ex(units=bad_u) == EINVAL and ex(merge=0.0) == EINVAL and ex(K=0) == EINVAL and ex(grid=None) == EINVAL
    assert ex(n_points=4097) == ENOSPACE


def test_extract_tracks_rejects():
    g = _grid()
    call = lambda n_points, merge, K, R0=1.0: L.retina_extract_tracks(
        BOGUS, BOGUS, None, None, 1, n_points, ctypes.byref(g), R0, merge, BOGUS, BOGUS, None, BOGUS, K, None)
    assert call(8193, 2.0, 8) == ENOSPACE
    assert call(16, 0.0, 8) == EINVAL
    assert call(16, float("nan"), 8) == EINVAL
    assert call(16, 2.0, 0) == EINVAL
    assert call(16, 2.0, 8, R0=float("nan")) == EINVAL
    assert call(16, 1e-3, 8) == EINVAL  # too many merge buckets per axis


def test_response_rejects():
    assert L.retina_response(BOGUS, 10, BOGUS, 1, 1, BOGUS, 4, 0.0, 1, BOGUS, None) == EINVAL
    assert L.retina_response(BOGUS, 10, BOGUS, 1, 5, BOGUS, 4, 0.3, 1, BOGUS, None) == EINVAL
    assert L.retina_response(BOGUS, 10, BOGUS, 1, 1, None, 4, 0.3, 1, BOGUS, None) == EINVAL


def test_prepare_hits_rejects_and_counts():
    assert L.retina_prepare_hits_box_count(100, 3) == 100 // 32 + 3 + 1
    assert L.retina_prepare_hits(BOGUS, 10, BOGUS, 1, 5, BOGUS, BOGUS, None) == EINVAL  # model
    assert L.retina_prepare_hits(BOGUS, 10, BOGUS, 1, 1, BOGUS, BOGUS, None) == EINVAL  # in place
    assert L.retina_prepare_hits(BOGUS, 10, BOGUS, 1, 1, ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3004),
                                 None) == EINVAL  # misaligned boxes


def test_seednet_entries_reject_before_launch():
    OK = 0
    # slope histogram: range, zmin, nulls; empty batch is a no-op
    assert L.retina_slope_histogram(BOGUS, 10, BOGUS, 1, 0.5, -0.5, 50.0, BOGUS, None, None) == EINVAL
    assert L.retina_slope_histogram(BOGUS, 10, BOGUS, 1, -0.5, 0.5, -1.0, BOGUS, None, None) == EINVAL
    assert L.retina_slope_histogram(BOGUS, 10, BOGUS, 1, float("nan"), 0.5, 50.0, BOGUS, None, None) == EINVAL
    assert L.retina_slope_histogram(BOGUS, 10, BOGUS, 1, -0.5, 0.5, 50.0, None, None, None) == EINVAL
    assert L.retina_slope_histogram(ctypes.c_void_p(0x1004), 10, BOGUS, 1, -0.5, 0.5, 50.0, BOGUS, None, None) == EINVAL
    assert L.retina_slope_histogram(None, 0, None, 0, -0.5, 0.5, 50.0, None, None, None) == OK
    # forward: h1 is required
    assert L.retina_seednet_forward(BOGUS, 1, BOGUS, BOGUS, None, None, None) == EINVAL
    assert L.retina_seednet_forward(BOGUS, -1, BOGUS, BOGUS, BOGUS, None, None) == EINVAL
    assert L.retina_seednet_forward(None, 0, None, None, None, None, None) == OK
    # training step: Adam hyper-parameters, step, workspace
    b = ctypes.c_size_t()
    assert L.retina_seednet_train_workspace_size(4, ctypes.byref(b)) == OK and b.value > 4 * 4096 * 48
    args = lambda **k: [k.get("feat", BOGUS), BOGUS, k.get("E", 4), BOGUS, BOGUS, BOGUS, k.get("step", 1),
                        k.get("lr", 1e-3), k.get("b1", 0.9), k.get("b2", 0.999), k.get("eps", 1e-8), None, None,
                        k.get("ws", ctypes.c_void_p(0x10000)), k.get("wsb", b.value), None]
    assert L.retina_seednet_train_step(*args(step=0)) == EINVAL
    assert L.retina_seednet_train_step(*args(b1=1.0)) == EINVAL
    assert L.retina_seednet_train_step(*args(b2=0.0)) == EINVAL
    assert L.retina_seednet_train_step(*args(lr=float("inf"))) == EINVAL
    assert L.retina_seednet_train_step(*args(E=0)) == EINVAL
    assert L.retina_seednet_train_step(*args(feat=None)) == EINVAL
    assert L.retina_seednet_train_step(*args(wsb=b.value - 1)) == ENOSPACE
    assert L.retina_seednet_train_step(*args(ws=ctypes.c_void_p(0x10010))) == EINVAL  # not 256-byte aligned
    assert L.retina_seednet_adam(BOGUS, BOGUS, BOGUS, BOGUS, 0, 1e-3, 0.9, 0.999, 1e-8, None) == EINVAL
    assert L.retina_seednet_adam(BOGUS, BOGUS, None, BOGUS, 1, 1e-3, 0.9, 0.999, 1e-8, None) == EINVAL
    # top-K: K range, box, n_min, hits without offsets
    T = lambda *a: L.retina_topk_seeds(*a)
    assert T(BOGUS, 1, 0, -0.5, 0.5, 50.0, 3, None, 0, None, BOGUS, None, None) == EINVAL
    assert T(BOGUS, 1, 4097, -0.5, 0.5, 50.0, 3, None, 0, None, BOGUS, None, None) == EINVAL
    assert T(BOGUS, 1, 16, 0.5, 0.5, 50.0, 3, None, 0, None, BOGUS, None, None) == EINVAL
    assert T(BOGUS, 1, 16, -0.5, 0.5, 50.0, 0, None, 0, None, BOGUS, None, None) == EINVAL
    assert T(BOGUS, 1, 16, -0.5, 0.5, -1.0, 3, None, 0, None, BOGUS, None, None) == EINVAL
    assert T(BOGUS, 1, 16, -0.5, 0.5, 50.0, 3, None, 0, None, None, None, None) == EINVAL
    assert T(BOGUS, 1, 16, -0.5, 0.5, 50.0, 3, BOGUS, 10, None, BOGUS, None, None) == EINVAL
    assert T(ctypes.c_void_p(0x1004), 1, 16, -0.5, 0.5, 50.0, 3, None, 0, None, BOGUS, None, None) == EINVAL  # logits
    assert T(None, 0, 16, -0.5, 0.5, 50.0, 3, None, 0, None, None, None, None) == OK


def test_sort_seeds_rejects_before_launch():
    g = rt.Grid((-0.5, -0.5), (2 ** -10, 2 ** -10), (1024, 1024)).c()
    bad = rt.Grid((-0.5, -0.5), (0.0, 2 ** -10), (1024, 1024)).c()
    assert L.retina_sort_seeds(BOGUS, 10, BOGUS, 1, ctypes.byref(bad), ctypes.c_void_p(0x2000), None, None) == EINVAL
    assert L.retina_sort_seeds(BOGUS, 10, BOGUS, 1, ctypes.byref(g), BOGUS, None, None) == EINVAL  # in place
    assert L.retina_sort_seeds(ctypes.c_void_p(0x1004), 10, BOGUS, 1, ctypes.byref(g), ctypes.c_void_p(0x2000),
                               None, None) == EINVAL  # misaligned
    assert L.retina_sort_seeds(None, 0, None, 0, ctypes.byref(g), None, None, None) == 0


def test_pipeline_config_validation_needs_no_gpu():
    import ctypes

    def cfg(**kw):
        c = rt._CPipelineConfig()
        c.model, c.grid, c.sigma_grid, c.R0, c.merge_cells = 1, _grid(), 0.378, 11.7, 2.0
        c.opts = rt.LsOpts().c()
        c.max_events, c.max_hits, c.seeds_per_event, c.max_maxima, c.max_tracks = 1, 4096, 8192, 8192, 4096
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    h = ctypes.c_void_p()
    bad = [dict(model=7), dict(sigma_grid=0.0), dict(R0=float("nan")), dict(merge_cells=-1.0),
           dict(max_events=0), dict(max_hits=-1), dict(seeds_per_event=0), dict(seeds_per_event=8193),
           dict(max_maxima=0), dict(max_maxima=9000), dict(max_tracks=0), dict(merge_cells=1e-3)]
    for kw in bad:
        assert L.retina_pipeline_create(ctypes.byref(cfg(**kw)), ctypes.byref(h)) == EINVAL, kw
        assert h.value is None
    c = cfg()
    c.opts.q = 0
    assert L.retina_pipeline_create(ctypes.byref(c), ctypes.byref(h)) == EINVAL
    assert L.retina_pipeline_create(None, ctypes.byref(h)) == EINVAL
    assert L.retina_pipeline_create(ctypes.byref(cfg()), None) == EINVAL
    assert L.retina_pipeline_destroy(None) == EINVAL
    assert L.retina_pipeline_run(None, None, 0, None, 1, None, None, None, None, None, None, None, None) == EINVAL


def test_option_structs_marshal_every_field():
    o = rt.LsOpts(sigma=(0.4, 0.2), c1=0.25, max_halvings=5, step_cap_cells=2.5, update=rt.UPDATE_MODIFIED_NEWTON).c()
    assert (o.q, list(o.sigma)[:2], o.max_halvings, o.update) == (2, [pytest.approx(0.4), pytest.approx(0.2)], 5, 2)
    assert o.c1 == pytest.approx(0.25) and o.step_cap_cells == pytest.approx(2.5)
    r = rt.refine_opts(0.378, iters=3, step_cap_cells=0.5)
    assert r.sigma == (0.378,) * 3 and r.step_cap_cells == 0.5 and r.update == rt.UPDATE_TRUNCATED_NEWTON
    f = rt.LsOpts4(sigma=(0.3, 0.05), scale=(0.25, 0.5, 1e-3, 2e-3), step_cap=3.0, zref=225.0).c()
    assert f.q == 2 and list(f.scale) == [pytest.approx(v) for v in (0.25, 0.5, 1e-3, 2e-3)]
    assert f.step_cap == pytest.approx(3.0) and f.zref == pytest.approx(225.0)
    # the C struct sizes the library expects (host pointers read field by field)
    assert ctypes.sizeof(type(f)) == 4 * (1 + 8 + 1 + 1 + 4 + 1 + 1)


def test_tracker_configuration_is_validated_before_allocating():
    good = rt._CTrackerConfig()
    good.box = rt.Grid((-0.5, -0.5), (2 ** -10, 2 ** -10), (1024, 1024)).c()
    good.opts = rt.LsOpts().c()
    good.R0, good.merge_cells = 11.7, 2.0
    good.max_events, good.max_hits, good.seeds_per_event, good.max_tracks = 4, 1000, 512, 64
    good.use_graph = 1
    h = ctypes.c_void_p()
    assert L.retina_tracker_create(None, None, ctypes.byref(h)) == EINVAL
    for field, value in (("max_events", 0), ("max_events", 65536), ("seeds_per_event", 0),
                         ("seeds_per_event", 8193), ("max_tracks", 0), ("max_hits", -1), ("sort_seeds", 2),
                         ("seeds_per_warp", 3), ("warps", 12), ("smem_hits", 12289), ("merge_cells", 0.0),
                         ("R0", float("nan"))):
        c = rt._CTrackerConfig.from_buffer_copy(good)
        setattr(c, field, value)
        assert L.retina_tracker_create(ctypes.byref(c), None, ctypes.byref(h)) == EINVAL, field
        assert not h.value
    c = rt._CTrackerConfig.from_buffer_copy(good)
    c.opts.q = 0
    assert L.retina_tracker_create(ctypes.byref(c), None, ctypes.byref(h)) == EINVAL
    assert L.retina_tracker_step(None, 1, None) == EINVAL
    assert L.retina_tracker_run_host(None, None, 0, None, 1, None, None, None, None, None) == EINVAL
    assert L.retina_tracker_destroy(None) == EINVAL


def test_extract_tracks_ws_sizes_and_validation():
    b = ctypes.c_size_t()
    assert L.retina_extract_tracks_workspace_size(4, 8192, ctypes.byref(b)) == 0 and b.value == 0
    assert L.retina_extract_tracks_workspace_size(4, 8193, ctypes.byref(b)) == 0 and b.value >= 4 * 16384 * 17
    assert L.retina_extract_tracks_workspace_size(4, (1 << 22) + 1, ctypes.byref(b)) == EINVAL
    g = _grid()
    args = (BOGUS, BOGUS, None, None, 2, 20000, ctypes.byref(g), 5.0, 2.0, BOGUS, BOGUS, None, BOGUS, 8)
    need = ctypes.c_size_t()
    L.retina_extract_tracks_workspace_size(2, 20000, ctypes.byref(need))
    assert L.retina_extract_tracks_ws(*args, WS, need.value - 1, None) == ENOSPACE
    assert L.retina_extract_tracks_ws(*args, ctypes.c_void_p(0x2010), need.value, None) == EINVAL  # misaligned
    assert L.retina_extract_tracks_ws(*args, None, need.value, None) == EINVAL
    assert L.retina_extract_tracks(*args, None) == ENOSPACE  # the shared-memory form stops at 8192
