"""Consistent cut across ranks (one process per GPU).

The paper checkpoints MPI applications by quiescing every rank and the
network before the per-process checkpoints are taken (Section 3.3: each MPI
process drains its GPU and a child of each process writes the image;
Section 4.5: quiescing and draining in-flight messages cost 0.01 % of the
total).  On this path each rank checkpoints its own registered set, so a
cut needs only host coordination: every rank stops sending, meets the
others at a barrier, then takes its checkpoint; an all-gather of each
rank's cut number and outcome decides, identically on every rank, whether
the cut stands.  Restoring a cut is the same: an agreement that every rank
holds an image of that cut, a barrier, each rank's restore, a barrier.

Rules (the same decision on every rank, from the gathered values only):

* A cut stands when every rank is at the same cut number and every rank's
  checkpoint call succeeded (the image was queued; its capture is the
  rank's consistency point).  The cut is named by that number; each rank
  keeps its own image of it.
* Otherwise the cut is refused on every rank.  Each rank drops its handle of
  the refused cut's image.  An image that was captured stays a link of its
  rank's chain (it holds that rank's state at that moment, so restoring a
  later cut through it is exact); a rank whose checkpoint failed gets a full
  image at its next checkpoint when the library marked its set so (a failed
  capture does).
* Cut numbers continue from one past the largest any rank held, so ranks
  that were out of step (one a cut ahead) are in step for the next cut.
* A rank that does not reach a cut (it left, or stalled beyond the
  coordinator's timeout) is detected on the host, by the barrier or the
  all-gather failing, before any rank queues device work for that cut or
  after it has queued only its own capture: the others raise RankLost and
  drop their image of that cut.

Host logic only (torch.distributed); the device work is each rank's own
crum_checkpoint / crum_restore.
"""
from __future__ import annotations

from typing import Any, Dict, Optional

__all__ = ["CutError", "RankLost", "CutCoordinator"]


class CutError(RuntimeError):
    pass


class RankLost(CutError):
    """A rank did not reach the cut (it left, or its host stalled beyond the
    timeout): the cut is abandoned on every rank that noticed."""


def _gather(values, group) -> list:
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.tensor(list(values), dtype=torch.int64)
    out = [torch.zeros(len(values), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return [[int(v) for v in x.tolist()] for x in out]


class CutCoordinator:
    """One rank's side of the cut protocol over its checkpoint set.

    `cset` needs ``checkpoint(stream, flags) -> image`` and
    ``restore(image, stream)``; images need ``info() -> {"seq": ...}`` and
    ``release()``."""

    def __init__(self, cset: Any, group: Optional[Any] = None, first_cut: int = 0,
                 timeout_s: Optional[float] = None):
        self.cset = cset
        self.group = group
        self.next_cut = first_cut
        self.timeout_s = timeout_s  # how long a barrier waits for every rank
        self.images: Dict[int, Any] = {}   # cut number -> this rank's image
        self.seqs: Dict[int, list] = {}    # cut number -> every rank's image seq

    def _barrier(self) -> None:
        """Every rank arrives, or RankLost.  With a timeout on a gloo group
        the barrier is monitored: it names the ranks that did not arrive."""
        import datetime
        import torch.distributed as dist
        try:
            if self.timeout_s is not None and dist.get_backend(self.group) == "gloo":
                dist.monitored_barrier(self.group, timeout=datetime.timedelta(seconds=self.timeout_s))
            else:
                dist.barrier(self.group)
        except RuntimeError as e:
            raise RankLost(f"a rank did not reach the cut: {e}") from e

    def _gather(self, values) -> list:
        try:
            return _gather(values, self.group)
        except RuntimeError as e:  # a peer left between the barrier and here
            raise RankLost(f"a rank left during the cut: {e}") from e

    def checkpoint(self, stream: int, flags: int = 0):
        """Barrier, this rank's checkpoint, agreement.  Returns (image, cut
        number); raises CutError on every rank when the cut is refused, and
        RankLost when a rank does not take part (this rank's image, if it
        took one, is dropped: the cut cannot stand)."""
        self._barrier()
        img, err = None, ""
        try:
            img = self.cset.checkpoint(stream, flags)
        except Exception as e:  # the rank reports the failure instead of leaving
            err = str(e)
        seq = int(img.info()["seq"]) if img is not None else -1
        try:
            rows = self._gather([self.next_cut, int(img is not None), seq])
        except RankLost:
            if img is not None:
                img.release()
            raise
        cuts = [r[0] for r in rows]
        ok = len(set(cuts)) == 1 and all(r[1] for r in rows)
        self.next_cut = max(cuts) + 1
        if not ok:
            if img is not None:
                img.release()
            why = (f"ranks are at different cuts: {cuts}" if len(set(cuts)) != 1 else
                   f"checkpoint failed on ranks {[i for i, r in enumerate(rows) if not r[1]]}")
            raise CutError(why + (f" (this rank: {err})" if err else ""))
        cut = cuts[0]
        self.images[cut] = img
        self.seqs[cut] = [r[2] for r in rows]
        return img, cut

    def restore(self, cut: int, stream: int, wait=None) -> int:
        """Every rank restores its image of cut `cut`; refused on every rank
        unless all ranks hold one.  `wait` (a callable, e.g. a stream
        synchronize) runs after the stream-ordered restore is queued and
        before the closing barrier, so that the barrier means every rank's
        memory is back."""
        mine = self.images.get(cut)
        rows = self._gather([cut, int(mine is not None)])
        if len({r[0] for r in rows}) != 1 or not all(r[1] for r in rows):
            raise CutError(f"not every rank holds an image of cut {cut}: {rows}")
        self._barrier()
        self.cset.restore(mine, stream)
        if wait is not None:
            wait()
        self._barrier()
        return cut

    def release(self) -> None:
        for img in self.images.values():
            img.release()
        self.images.clear()
