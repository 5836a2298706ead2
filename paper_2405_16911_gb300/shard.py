"""Splitting one long stream over several GPUs (one process per GPU).

Because the phase uses the absolute sample index, contiguous time segments can be
estimated independently: rank r commits the terms n in [a_r, b_r) of the whole stream
by pushing samples [a_r, b_r + M) into a stream created with start index n0 + a_r.  Its
estimate R_r (over N_r = b_r - a_r terms) and the others combine exactly by

    R = sum_r N_r R_r / sum_r N_r

which is one SUM reduction of F*A*L complex FP64 values (and the counts) at read time:
allreduce_stream() adds the ranks' libcyc running sums in place on the device (NCCL) and
sets the merged count, so that the library's own read divides by it.  Independent streams
(serving) need no exchange at all.
"""
from __future__ import annotations

import numpy as np

__all__ = ["time_shards", "merge", "allreduce_merge", "allreduce_stream"]


def time_shards(T: int, M: int, world: int):
    """[(sample_start, sample_end, n_start, n_count)] per rank for a stream of T samples
    and max lag M: the committed ranges [n_start, n_start + n_count) partition [0, T - M)
    and rank r reads samples [sample_start, sample_end) = [n_start, n_start + n_count + M)."""
    if world < 1 or T < 0 or M < 0:
        raise ValueError("bad shard request")
    n_total = max(0, T - M)
    out = []
    for r in range(world):
        a = r * n_total // world
        b = (r + 1) * n_total // world
        out.append((a, b + M if b > a else a, a, b - a))
    return out


def merge(results):
    """Combine [(R_r, N_r)] into (R, N): the N-weighted mean of the shard estimates."""
    num = None
    n = 0
    for R, N in results:
        if N <= 0:
            continue
        num = R * N if num is None else num + R * N
        n += N
    if n == 0:
        return None, 0
    return num / n, n


def allreduce_merge(R_local, n_local: int, group=None):
    """The same combination across ranks with one torch.distributed SUM (gloo or NCCL):
    every rank receives the merged estimate and the total count."""
    import torch
    import torch.distributed as dist
    if R_local is None:
        raise ValueError("R_local must be an array of the stream's output shape (zeros if N = 0)")
    R = np.asarray(R_local, dtype=np.complex128)
    buf = np.concatenate([(R * n_local).view(np.float64).ravel(), [float(n_local)]])
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.from_numpy(buf).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    out = t.cpu().numpy()
    n = int(round(out[-1]))
    if n == 0:
        return None, 0
    Rm = out[:-1].view(np.complex128).reshape(R.shape) / n
    return Rm, n


def allreduce_stream(stream, group=None) -> int:
    """Merge the time shards held by every rank's libcyc stream (same parameters, start index
    of its shard): one in-place SUM all-reduce of the stream's FP64 device sums and one of the
    counts; afterwards stream.read() returns the whole stream's estimate.  Returns N_eff."""
    import torch
    import torch.distributed as dist
    sums, n = stream.sums()
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    cnt = torch.tensor([n], dtype=torch.int64, device=sums.device)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM, group=group)
    total = int(cnt.item())                 # waits for both reductions (one NCCL stream, in order)
    torch.cuda.synchronize()
    stream.set_n_eff(total)
    return total
