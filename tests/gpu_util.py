"""Helpers for the GPU tests: numpy <-> torch conversions of the uint16 planes,
and the comparison of an encode's buffers with the oracle's outputs."""
import numpy as np
import torch


def to_np(t):
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def to_dev(a, device="cuda"):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).to(device).view(torch.uint16)
    return torch.from_numpy(a).to(device)


def assert_matches(buf, res, want, frames=None):
    """Every output of one encode equal to the oracle's (PSNR within 1e-9
    relative); with `frames`, only those first frames (copied from the device
    alone) and no cube totals."""
    sl = slice(None) if frames is None else slice(0, frames)
    assert np.array_equal(to_np(buf["planes"][:, sl]), want["planes"][:, sl])
    assert np.array_equal(to_np(buf["mv"][:, sl]), want["mv"][:, sl])
    assert np.array_equal(to_np(buf["cost"][:, sl]).astype(np.uint32), want["cost"][:, sl])
    assert np.array_equal(to_np(buf["recon"][:, sl]), want["recon"][:, sl])
    assert np.array_equal(to_np(buf["levels"][:, sl]), want["levels"][:, sl])
    assert np.array_equal(to_np(buf["tu_log2"][:, sl]), want["tu_log2"][:, sl])
    assert np.array_equal(to_np(buf["bits"][:, sl]).astype(np.uint64), want["bits"][:, sl])
    if frames is None:
        assert res["total_bits"] == want["total_bits"]
        for g, w in zip(res["psnr_band"], want["psnr_band"]):
            assert (np.isinf(g) and np.isinf(w)) or abs(g - w) <= 1e-9 * abs(w)
        assert res["sse10_band"] == [int(v) for v in want["sse10_band"]]
