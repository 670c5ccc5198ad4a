"""Rule split across GPUs: each rank holds one contiguous range of the rule list.

The function-parallel and hybrid designs (Sec. IV.B, IV.C) split the rule list
over workers and combine their results. Inside one GPU the rule-split kernels
do that with warp votes and atomic minima; across GPUs the same combine takes
one exchange. Every rank classifies all packets against its own range and
turns its first match into a global rule index (NO_MATCH when its range holds
none). An elementwise minimum over the ranks (all_reduce MIN) then gives each
packet's first match in the whole list: the first match in a union of
consecutive ranges is the smallest of their first matches (Sec. I, first
match). The action of that rule comes from the action table every rank holds;
no rule matching means DROP (default deny).

Ranks are torch.distributed ranks (NCCL between GPUs, gloo on CPU); with one
rank, or no process group, the combine is the identity. Classification runs in
the CUDA library (fw_classify on the rank's range); the index remap, the
minimum and the action lookup are elementwise tensor operations on the current
stream.
"""
from __future__ import annotations

import numpy as np

NO_MATCH = 2**31 - 1  # int32 max: no rule of this range matches


def shard_range(n_rules: int, world: int, rank: int) -> tuple[int, int]:
    """Rules [lo, hi) of rank ``rank``: contiguous ranges in rank order, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_rules < 0:
        raise ValueError(f"bad shard: n_rules={n_rules} world={world} rank={rank}")
    q, r = divmod(int(n_rules), int(world))
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def to_global(local_idx, lo: int):
    """Range-local first match (-1 = none) to a global rule index (NO_MATCH = none), int32."""
    import torch
    return torch.where(local_idx >= 0, local_idx + int(lo), torch.full_like(local_idx, NO_MATCH))


def combine(global_idx, group=None):
    """Elementwise minimum of ``global_idx`` over the ranks of ``group``, in place; returns it."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(global_idx, op=dist.ReduceOp.MIN, group=group)
    return global_idx


def finalize(global_idx, actions):
    """(rule index, -1 where no range matched; the rule's action, DROP (0) where none)."""
    import torch
    none = global_idx == NO_MATCH
    idx = torch.where(none, torch.full_like(global_idx, -1), global_idx)
    if actions.numel() == 0:
        return idx, torch.zeros(idx.shape, dtype=torch.uint8, device=idx.device)
    act = actions[idx.clamp(min=0).long()]
    return idx, torch.where(none, torch.zeros_like(act), act)


class RuleShard:
    """This rank's range of the rule list as a CUDA rule set, and the whole list's action table."""

    def __init__(self, rules, world: int, rank: int, device="cuda"):
        import torch

        from . import fw
        self.lo, self.hi = shard_range(len(rules), world, rank)
        self.rs = fw.fw_ruleset_create(rules[self.lo:self.hi])
        self.actions = torch.as_tensor(np.ascontiguousarray(rules["action"]).astype(np.uint8), device=device)

    def classify(self, hdrs: dict, n: int | None = None, group=None):
        """First match in the whole list for every packet (same headers on every rank): (idx, action)."""
        from . import fw
        local, _ = fw.fw_classify(self.rs, hdrs, n)
        return finalize(combine(to_global(local, self.lo), group), self.actions)

    def destroy(self):
        if self.rs is not None:
            self.rs.destroy()
        self.rs = None
