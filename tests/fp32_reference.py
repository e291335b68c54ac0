"""The same operators written in plain PyTorch FP32 (rfft2 / irfft2) on the GPU:
the FP32 error bar for white-noise inputs, whose solutions sit in the lowest bins
where any FP32 transform's round-off is amplified by |G| ~ (M / 2 pi)^2. Tests
hold the library to max(1e-5, 3 x the error of these) on such inputs."""
import numpy as np
import torch

import oracle.gfc_oracle as O


def torch_fp32_adjoint(gout, M, N, p, dev):
    """Adjoint of the solve (Crop^T, minus the sum at (0, 0), Green multiply, -D)."""
    H, W = gout.shape
    G = torch.from_numpy(O.green_spectrum(M, N)[:, : N // 2 + 1]).float().to(dev)
    z = torch.zeros((M, N), device=dev)
    g = torch.from_numpy(np.ascontiguousarray(gout, dtype=np.float32)).to(dev)
    z[p:p + H, p:p + W] = g
    z[0, 0] -= g.sum()
    w = torch.fft.irfft2(torch.fft.rfft2(z) * G, s=(M, N))
    gx = (w - torch.roll(w, -1, -1))[p:p + H, p:p + W]
    gy = (w - torch.roll(w, -1, -2))[p:p + H, p:p + W]
    return gx.double().cpu().numpy(), gy.double().cpu().numpy()


def torch_fp32_laplacian_solve(lap, M, N, p, dev):
    """Solve from a Laplacian (mean removed by G[0,0] = 0), offset u[0,0], crop."""
    H, W = lap.shape
    G = torch.from_numpy(O.green_spectrum(M, N)[:, : N // 2 + 1]).float().to(dev)
    L = torch.zeros((M, N), device=dev)
    L[p:p + H, p:p + W] = torch.from_numpy(np.ascontiguousarray(lap, dtype=np.float32)).to(dev)
    u = torch.fft.irfft2(torch.fft.rfft2(L) * G, s=(M, N))
    return (u - u[0, 0])[p:p + H, p:p + W].double().cpu().numpy()
