"""Data-parallel use of the chemistry substep over several GPUs (one process
per GPU).  Cells are independent (Sec. 2.3: every cell integrates its own
kinetics ODE), so the integrator and the DNN inference shard by cell ranges
with no collective.  Two steps do exchange data:

* the adjoint's gradient with respect to ln A is a sum over cells: one
  all-reduce of M doubles after each rank's df_chem_adjoint on its own cells;
* DNN training (the paper names multi-card DNN work as future work, Sec. 6)
  is data-parallel: each rank runs df_dnn_grad on its shard of the batch,
  normalised by the global row count, the ranks sum the FP32 gradient buffers
  in place, and each runs df_dnn_adam_step, so every rank keeps the same
  parameters.

Arithmetic stays in the library's kernels and in the collective; this module
only partitions and orchestrates.  The collective is torch.distributed
(NCCL on GPUs; with gloo the buffers travel through host memory).
"""
from __future__ import annotations

import numpy as np


def partition(ncells: int, world: int, work=None):
    """Contiguous cell ranges [(lo, hi)] for `world` ranks.  Without `work`
    the ranges differ in size by at most one cell; with `work` (a per-cell cost
    estimate, e.g. the previous step's substep counts) each range gets about
    the same total work, so ranks of uneven stiffness finish together."""
    if world < 1 or ncells < 0:
        raise ValueError("partition: world >= 1 and ncells >= 0")
    if work is None:
        cuts = [(ncells * r) // world for r in range(world + 1)]
    else:
        w = np.asarray(work, dtype=np.float64)
        if w.shape != (ncells,) or np.any(w < 0) or not np.all(np.isfinite(w)):
            raise ValueError("partition: work must be ncells finite values >= 0")
        cum = np.concatenate([[0.0], np.cumsum(w)])
        total = cum[-1]
        cuts = [0]
        for r in range(1, world):
            c = int(np.searchsorted(cum, total * r / world, side="left"))
            cuts.append(min(max(c, cuts[-1]), ncells))
        cuts.append(ncells)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def allreduce_sum_(t, group=None):
    """Sum a tensor over the ranks of `group` in place.  With a CPU-only
    backend (gloo) a CUDA tensor goes through a host copy."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return t
    backend = dist.get_backend(group)
    if t.is_cuda and backend == "gloo":
        h = t.detach().cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        t.copy_(h.to(t.device))
        torch.cuda.current_stream(t.device).synchronize()
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def dp_train_step(dnn, T, p, Y, Y_next, lr: float, n_total: int, group=None, want_loss: bool = True):
    """One data-parallel Adam step: this rank's rows (T, p, Y, Y_next) are its
    shard of a global batch of n_total rows.  Returns the global loss (the sum
    of the ranks' shares) when want_loss."""
    loss = dnn.grad(T, p, Y, Y_next, n_total=n_total, want_loss=want_loss)
    allreduce_sum_(dnn.grad_tensor(), group)
    dnn.adam_step(lr)
    if want_loss:
        import torch
        lt = torch.tensor([float(loss)], dtype=torch.float64)
        allreduce_sum_(lt, group)
        return float(lt.item())
    return None


def adjoint_sharded(mech, T0, p, Y0, dt: float, gT1=None, gY1=None, gQ1=None, opts=None, max_steps: int = 64,
                    group=None):
    """df_chem_adjoint on this rank's cells, then the ln A gradient summed over
    the ranks (one all-reduce of M doubles).  gT0, gY0 stay per cell."""
    from . import adjoint
    out = adjoint(mech, T0, p, Y0, dt, gT1, gY1, gQ1, opts, max_steps)
    allreduce_sum_(out["g_lnA"], group)
    return out
