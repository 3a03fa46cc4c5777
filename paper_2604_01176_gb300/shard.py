"""Row distribution of H|psi> over processes.

The paper distributes the Hamiltonian only: its rows, the determinants of
Omega_CIk, are split uniformly over the processes and the state vector is
replicated on each; every process forms the components of its own rows, and
one collective completes the operation -- an all-gather (broadcast) of the
row blocks, or an all-reduce of the scalars formed from them (Sparse
State-Vector Emulation section, parallelisation paragraph).

Here a row is an alpha string (N_beta consecutive determinants), the
library's hy_apply_h_rows forms a block and hy_dot_rows its partial inner
products; this module holds the split and the two collectives, written once
for any torch.distributed backend (NCCL between GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def row_split(n_rows: int, world: int, rank: int) -> tuple[int, int]:
    """Uniform contiguous split of n_rows over `world` processes: rank r owns
    [r * n_rows // world, (r + 1) * n_rows // world)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    return rank * n_rows // world, (rank + 1) * n_rows // world


def gather_blocks(block: torch.Tensor, n_rows: int, n_cols: int, group=None) -> torch.Tensor:
    """All-gather the row blocks of every process into the full vector of
    n_rows * n_cols elements (blocks are uneven by at most one row: each is
    padded to the largest, gathered, and trimmed)."""
    world = dist.get_world_size(group)
    spans = [row_split(n_rows, world, r) for r in range(world)]
    widest = max(e - b for b, e in spans) * n_cols
    pad = torch.zeros(widest, dtype=block.dtype, device=block.device)
    pad[: block.numel()] = block.reshape(-1)
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[: (e - b) * n_cols] for p, (b, e) in zip(parts, spans)])


def reduce_partials(partials: torch.Tensor, group=None) -> torch.Tensor:
    """Sum FP64 per-process partial scalars over the processes (in place)."""
    if partials.dtype != torch.float64:
        raise TypeError("partials must be float64")
    dist.all_reduce(partials, op=dist.ReduceOp.SUM, group=group)
    return partials


def sharded_apply_h(ham, psi: torch.Tensor, group=None) -> torch.Tensor:
    """sigma = H psi with this process forming its rows (hy_apply_h_rows)
    and one all-gather assembling the whole vector on every process."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    b, e = row_split(ham.n_alpha_str, world, rank)
    block = ham.apply_h_rows(psi, b, e)
    return gather_blocks(block, ham.n_alpha_str, ham.n_beta_str, group)


def sharded_energy(ham, psi: torch.Tensor, group=None) -> torch.Tensor:
    """<psi|H|psi> from this process's rows: its block of sigma, the partial
    <psi_rows|sigma_rows> (hy_dot_rows, FP64) and one all-reduce."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    b, e = row_split(ham.n_alpha_str, world, rank)
    block = ham.apply_h_rows(psi, b, e)
    nb = ham.n_beta_str
    part = ham.dot_rows(psi[b * nb: e * nb], block, b, e).reshape(1)
    return reduce_partials(part, group)[0]
