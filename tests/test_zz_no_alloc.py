"""retina_grid_maxima_static: the grid-maxima selection for callers that cannot
allocate device memory (a plugin inside a host application whose memory
manager owns every device allocation, or a foreign-language caller with no
device allocator) and therefore cannot hand the library a workspace.  Its
scratch is a fixed library-owned device array.

The test calls it through the C ABI twice in a row, on different inputs, and
checks each result against retina_grid_maxima (which takes a caller
workspace) on the same input: the selection is integer work on identical
float32 inputs, so the tolerance used throughout the tests for such outputs
applies - exact equality.  A 2048 x 2048 case (2048 cell blocks per event,
more than one pass of the per-event scan) with fewer output slots than
maxima is also compared with the FP64 oracle's selection on the same values.
It checks that an input too large for the fixed scratch is refused with
RETINA_ENOSPACE and too many events with RETINA_EINVAL.  The file name makes
pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

EINVAL, ENOSPACE = 1, 3


@pytest.fixture(scope="module")
def rt():
    from paper_1709_08610_gb300 import build as rbuild
    rbuild.build()
    from paper_1709_08610_gb300 import retina
    return retina


def _field(E, n0, n1, seed):
    # smooth positive field with many local maxima (sum of random bumps)
    g = torch.Generator(device="cpu").manual_seed(seed)
    y = torch.arange(n1, dtype=torch.float32)[:, None]
    x = torch.arange(n0, dtype=torch.float32)[None, :]
    out = torch.zeros((E, n1, n0))
    for e in range(E):
        c = torch.rand((40, 2), generator=g) * torch.tensor([n0, n1])
        w = 2.0 + 10.0 * torch.rand(40, generator=g)
        a = 1.0 + 20.0 * torch.rand(40, generator=g)
        for k in range(40):
            out[e] += a[k] * torch.exp(-((x - c[k, 0]) ** 2 + (y - c[k, 1]) ** 2) / w[k] ** 2)
    return out.cuda()


def _static_call(rt, R, grid, R0, K):
    E = R.shape[0]
    out = dict(max_idx=torch.full((E, K), -7, dtype=torch.int32, device="cuda"),
               max_theta=torch.full((E, K, 2), -7.0, dtype=torch.float32, device="cuda"),
               max_R=torch.full((E, K), -7.0, dtype=torch.float32, device="cuda"),
               n_max=torch.full((E,), -7, dtype=torch.int32, device="cuda"))
    g = grid.c()
    rc = rt.lib.retina_grid_maxima_static(
        ctypes.c_void_p(R.data_ptr()), E, ctypes.byref(g), float(R0), ctypes.c_void_p(out["max_idx"].data_ptr()),
        ctypes.c_void_p(out["max_theta"].data_ptr()), ctypes.c_void_p(out["max_R"].data_ptr()),
        ctypes.c_void_p(out["n_max"].data_ptr()), K, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def _same(ref, got, K):
    n_ref = ref["n_max"].cpu().numpy()
    assert np.array_equal(n_ref, got["n_max"].cpu().numpy())
    for e, n in enumerate(n_ref):
        k = min(int(n), K)
        for key in ("max_idx", "max_theta", "max_R"):
            assert np.array_equal(ref[key][e, :k].cpu().numpy(), got[key][e, :k].cpu().numpy()), key


def test_static_scratch_maxima_match_workspace_entry_point_on_two_calls(rt):
    # first call: 3 events on a ragged 300 x 260 grid; second: 2 events of 1024^2
    cases = [(_field(3, 300, 260, 1), rt.Grid((-1.0, -1.0), (2 ** -7, 2 ** -7), (300, 260)), 2.0, 128),
             (_field(2, 1024, 1024, 2), rt.Grid((-0.5, -0.5), (2 ** -10, 2 ** -10), (1024, 1024)), 1.0, 64)]
    for R, grid, R0, K in cases:
        rc, got = _static_call(rt, R, grid, R0, K)
        assert rc == 0, rt.lib.retina_strerror(rc)
        ref = rt.grid_maxima(R, grid, R0, K)
        torch.cuda.synchronize()
        assert int(ref["n_max"].min()) >= 1
        _same(ref, got, K)


def test_static_scratch_2048_grid_scan_carry_and_truncation(rt):
    # 2048^2 cells = 2048 blocks of 2048 cells per event: the per-event scan
    # runs over two 1024-block chunks and carries the first chunk's total;
    # K below the number of maxima keeps the first K in cell-index order
    n = 2048
    # bumps on a noisy plateau above R0: local maxima all over the grid
    g = torch.Generator(device="cpu").manual_seed(9)
    R = _field(2, n, n, 3) + 1.0 + 1e-3 * torch.rand((2, n, n), generator=g).cuda()
    grid = rt.Grid((-0.5, -0.5), (2 ** -11, 2 ** -11), (n, n))
    R0, K = 0.5, 300
    for _ in range(2):
        rc, got = _static_call(rt, R, grid, R0, K)
        assert rc == 0, rt.lib.retina_strerror(rc)
        ref = rt.grid_maxima(R, grid, R0, K)
        torch.cuda.synchronize()
        _same(ref, got, K)
    Rh = R.cpu().numpy()
    for e in range(2):
        exp, cnt, _ = oracle.grid_maxima(Rh[e], R0, with_margin=True)
        assert cnt > K and int(got["n_max"][e]) == cnt
        # both chunks of the scan hold maxima
        assert exp.min() < 1024 * 2048 and exp.max() >= 1024 * 2048
        assert got["max_idx"][e].cpu().numpy().tolist() == exp[:K].tolist()


def test_static_scratch_refuses_inputs_beyond_its_size(rt):
    # 2 int32 per 2048-cell block per event: 100 events of 2048^2 need 1.6 MB > 1 MiB
    grid = rt.Grid((-0.5, -0.5), (2 ** -11, 2 ** -11), (2048, 2048))
    g = grid.c()
    dummy = torch.empty(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = rt.lib.retina_grid_maxima_static(p, 100, ctypes.byref(g), 1.0, p, p, p, p, 8, None)
    assert rc == ENOSPACE
    # more events than one launch dimension holds: refused before any launch
    small = rt.Grid((-0.5, -0.5), (0.25, 0.25), (4, 4)).c()
    rc = rt.lib.retina_grid_maxima_static(p, 65536, ctypes.byref(small), 1.0, p, p, p, p, 8, None)
    assert rc == EINVAL
