"""Standard MUSIC with a full eigendecomposition (Sec. II-B, Eq. 4-6): the comparison
method for the fast variants, on the same GPU.

R = X X^H / T and the scan and peak search run in this library's kernels (fm_covariance,
fm_spectrum / fm_spectrum_array, fm_peaks); the M x M Hermitian eigendecomposition of
Eq. 4 is a plain library call (torch.linalg.eigh, cuSOLVER), whose eigenvectors of the
K largest eigenvalues span the signal subspace.  This is the O(M^3) step the randomized
sketch of Alg. 1 / 2 replaces.
"""
from __future__ import annotations


def full_eig_music(ctx, X, K: int, theta0: float, step: float, L: int, pos_wl=None, stream=None):
    """X: (B, M, T) or (M, T) complex64 CUDA tensor.  Returns (P (B, L), U_K (B, M, K),
    peak_idx (B, K), peak_deg (B, K), n_peaks (B,)), all on the device, asynchronous on the
    current stream."""
    import torch
    R = ctx.covariance(X, stream=stream)
    _, V = torch.linalg.eigh(R)                 # ascending eigenvalues
    Uk = V[:, :, -K:].contiguous()              # signal subspace: the K largest
    if pos_wl is None:
        P = ctx.spectrum(Uk, theta0, step, L, stream=stream)
    else:
        P = ctx.spectrum_array(Uk, theta0, step, L, pos_wl=pos_wl, stream=stream)
    idx, deg, n = ctx.peaks(P, K, theta0, step, stream=stream)
    return P, Uk, idx, deg, n
