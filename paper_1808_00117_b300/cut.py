"""Consistent cut across ranks (one process per GPU).

The paper checkpoints MPI applications by quiescing every rank and the
network before the per-process checkpoints are taken (Section 3.3: each MPI
process drains its GPU and a child of each process writes the image;
Section 4.5: quiescing and draining in-flight messages cost 0.01 % of the
total).  On
this path each rank checkpoints its own registered set, so a cut needs only
host coordination: every rank stops sending, meets the others at a barrier,
then submits its checkpoint; the images' sequence numbers name the cut, and
all ranks must agree on it (a rank that skipped or repeated a checkpoint is
out of step and the cut is refused on every rank).  Restoring a cut is the
same: a barrier, each rank's restore, a barrier.

Host logic only (torch.distributed); the device work is each rank's own
crum_checkpoint / crum_restore.
"""
from __future__ import annotations

from typing import Any, Optional

__all__ = ["CutError", "checkpoint_cut", "restore_cut"]


class CutError(RuntimeError):
    pass


def _gather_int(value: int, group) -> list:
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.tensor([value], dtype=torch.int64)
    out = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return [int(x.item()) for x in out]


def checkpoint_cut(cset: Any, stream: int, flags: int = 0, group: Optional[Any] = None):
    """Barrier, then this rank's checkpoint.  Returns (image, cut) where cut
    is the image sequence number every rank agreed on.  Raises CutError (on
    every rank) if the ranks' sequence numbers differ."""
    import torch.distributed as dist
    dist.barrier(group)
    img = cset.checkpoint(stream, flags)
    seq = int(img.info()["seq"])
    seqs = _gather_int(seq, group)
    if len(set(seqs)) != 1:
        raise CutError(f"ranks are at different checkpoints: {seqs}")
    return img, seq


def restore_cut(cset: Any, image: Any, stream: int, group: Optional[Any] = None) -> int:
    """Every rank restores its image of the same cut.  Returns the cut."""
    import torch.distributed as dist
    seq = int(image.info()["seq"])
    seqs = _gather_int(seq, group)
    if len(set(seqs)) != 1:
        raise CutError(f"ranks would restore different cuts: {seqs}")
    dist.barrier(group)
    cset.restore(image, stream)
    dist.barrier(group)
    return seq
