"""The benchmark's host-side history ring (bench.HostHistory): uploads hand the device the
last H solutions newest first at every fill level and across the wrap, as the shifted
array it replaced did."""
import torch

from bench import HostHistory


def test_host_history_uploads_newest_first():
    H, n = 5, 3
    h = HostHistory(torch, H, n, pin=False)
    dst = torch.full((H, n), -1.0, dtype=torch.float64)
    for k in range(13):
        h.push_from(torch.full((n,), float(k), dtype=torch.float64))
        h.upload(dst)
        m = min(H, k + 1)
        assert h.count == m
        want = torch.tensor([[float(k - j)] * n for j in range(m)], dtype=torch.float64)
        assert torch.equal(dst[:m], want)
