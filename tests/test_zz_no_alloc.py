"""fm_spectrum_noalloc: the allocation-free variant of the spectrum scan.

Callers that cannot let the library allocate device memory (a front end with a
memory map fixed at start-up, or a framework that owns every allocation) use
this entry point; its scratch is a fixed array inside the library.  The test
calls it through the C ABI twice in a row, on two different grids and inputs,
and requires each result to equal fm_spectrum's bit for bit (the same kernels run
on the same descriptors).  It is collected last on purpose and runs equally alone in a fresh
process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def test_spectrum_noalloc_matches_fm_spectrum_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_07434_gb300 import binding, build
    build.build()
    ctx = binding.Context(device=0)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(512, 8, (-75.0, 0.01, 15001), 2), (200, 13, (-60.0, 0.05, 2401), 3)]
    try:
        for M, nc, (th0, st, L), nf in cases:
            rng = np.random.default_rng(M + nc)
            U = np.stack([np.linalg.qr(rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc)))[0]
                          for _ in range(nf)]).astype(np.complex64)
            Ud = torch.from_numpy(U).cuda()
            P_ref = ctx.spectrum(Ud, th0, st, L).cpu().numpy().astype(np.float64)
            P = torch.full((nf, L), -1.0, dtype=torch.float32, device="cuda")
            rc = binding.fm_spectrum_noalloc(Ud.data_ptr(), nf, M, nc, 0.5, binding.FmGrid(th0, st, L),
                                             P.data_ptr(), stream)
            assert rc == binding.FM_OK
            Pn = P.cpu().numpy().astype(np.float64)
            # the same kernels on the same descriptors: bit for bit; the message gives the
            # distance in the units of test_spectrum_parity's bound (8 u M ncols on 1/P)
            assert np.array_equal(Pn, P_ref), np.max(np.abs(1.0 / Pn - 1.0 / P_ref)) / (8 * U32 * M * nc)
        # sizes beyond the fixed scratch are rejected before any work
        Ud = torch.zeros((1, 64, 4), dtype=torch.complex64, device="cuda")
        P = torch.empty(70000, dtype=torch.float32, device="cuda")
        assert binding.fm_spectrum_noalloc(Ud.data_ptr(), 1, 64, 4, 0.5, binding.FmGrid(-90.0, 0.001, 65537),
                                           P.data_ptr(), stream) == binding.FM_ERR_INVALID_ARG
        assert binding.fm_spectrum_noalloc(Ud.data_ptr(), 65, 64, 4, 0.5, binding.FmGrid(-90.0, 1.0, 181),
                                           P.data_ptr(), stream) == binding.FM_ERR_INVALID_ARG
    finally:
        ctx.close()
