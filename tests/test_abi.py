"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
function include/fastmusic.h declares, and its struct layout matches the binding.
No compute call is made (there may be no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1911_07434_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastmusic.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.exported_symbols()) == names


def test_struct_layout_matches_header(lib):
    # sizes implied by the C declarations on an LP64 ABI
    assert ctypes.sizeof(binding.FmArray) == 24
    assert ctypes.sizeof(binding.FmGrid) == 24
    assert ctypes.sizeof(binding.FmParams) == 40
    assert binding.FmFrame.arr.offset == 24 and binding.FmFrame.grid.offset == 48
    assert binding.FmFrame.p.offset == 72
    assert ctypes.sizeof(binding.FmFrame) == 168


def _frame(M=64, T=200, K=3, l=13, t=1, method=2, L=1801, X=1, out=1):
    f = binding.FmFrame()
    f.X = X
    f.T = T
    f.ldx = T
    f.arr = binding.FmArray(M, 0.5)
    f.grid = binding.FmGrid(-90.0, 0.1, L)
    f.p = binding.FmParams(method, K, l, t, 0, 0, 0, 0, 0)
    f.P_out = f.peak_idx = f.peak_deg = f.n_peaks = out
    return f


def test_workspace_planning_is_host_only(lib):
    """fm_workspace_bytes validates and sizes on the host (no device needed)."""
    ok = binding.fm_workspace_bytes([_frame()])
    # R (64*64*8) + C, V (64*13*8 each) + U_s (64*3*8) + tables, each 256-aligned
    assert ok >= 64 * 64 * 8 + 2 * 64 * 13 * 8 + 64 * 3 * 8 + 1801 * 8
    two = binding.fm_workspace_bytes([_frame(), _frame()])
    assert two > ok and two < 2 * ok       # one shared grid table
    for bad in (_frame(K=14), _frame(l=65, M=128), _frame(M=1), _frame(method=0), _frame(L=0), _frame(X=0),
                _frame(out=0), _frame(t=9), _frame(M=2048)):
        assert binding.fm_workspace_bytes([bad]) == 0


def test_array_positions_are_validated_and_sized_on_the_host(lib):
    """fm_array.pos_wl (Sec. II-A, element positions in wavelengths): invalid positions
    (non-finite, beyond 4096 wavelengths) are refused before any launch, and a frame with
    positions plans one position table beside the uniform frame's workspace."""
    import numpy as np
    f = _frame()
    base = binding.fm_workspace_bytes([f])
    good = np.linspace(0.0, 40.0, 64)
    f.arr = binding.FmArray(64, 0.5, good.ctypes.data)
    with_pos = binding.fm_workspace_bytes([f])
    assert with_pos >= base + 64 * 8
    for bad in (np.full(64, np.nan), np.full(64, 5000.0), np.concatenate([good[:-1], [np.inf]])):
        f.arr = binding.FmArray(64, 0.5, bad.ctypes.data)
        assert binding.fm_workspace_bytes([f]) == 0
    # two frames with equal positions (different buffers) share one table
    g1, g2 = _frame(), _frame()
    p1, p2 = good.copy(), good.copy()
    g1.arr = binding.FmArray(64, 0.5, p1.ctypes.data)
    g2.arr = binding.FmArray(64, 0.5, p2.ctypes.data)
    both = binding.fm_workspace_bytes([g1, g2])
    p2[3] += 0.25
    assert binding.fm_workspace_bytes([g1, g2]) >= both + 64 * 8


def test_covariance_plan_follows_the_batch_shape(lib):
    """The covariance work plan is kept per host thread for a repeated batch shape (each
    frame's M and T); sizing a batch must not depend on which batch was sized before it.
    One M = 512 frame splits its tiles along T (partial-tile workspace), a 64-frame batch
    does not, and a frame whose T differs changes the split stages."""
    one = [_frame(M=512, T=1024, K=8, l=24, L=15001)]
    many = [_frame(M=512, T=1024, K=8, l=24, L=15001, X=4096 * (i + 1)) for i in range(64)]
    other_t = [_frame(M=512, T=1040, K=8, l=24, L=15001)]
    w1 = binding.fm_workspace_bytes(one)
    w64 = binding.fm_workspace_bytes(many)
    wt = binding.fm_workspace_bytes(other_t)
    assert w1 > 0 and w64 > 0 and wt > 0
    for _ in range(2):
        assert binding.fm_workspace_bytes(many) == w64
        assert binding.fm_workspace_bytes(one) == w1
        assert binding.fm_workspace_bytes(other_t) == wt
        assert binding.fm_workspace_bytes(one) == w1
    # the lone frame's split tiles need partial-tile workspace (at least 40 parts of
    # 128 x 128 complex) that the frames of a 64-frame batch do not: a frame's own share
    # is the step from 32 to 64 frames (the grid table is shared)
    w32 = binding.fm_workspace_bytes(many[:32])
    own = (w64 - w32) / 32
    assert w1 - own >= 40 * 128 * 128 * 8
