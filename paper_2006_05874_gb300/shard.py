"""Row sharding of the path across ranks (one process per GPU).

The method shards by rows of A.  Every per-row quantity stays on its rank; the
gradient of Eq. 1 needs one sum of d values (and of ||A x||^2) per pass,

    grad f(x) = sum_p A_p^T (A_p x - b_p) + nu^2 x,

and each sketch one sum of m x d values per level, S A = sum_p S_{:,p} A_p
(the SRHT over whole 1024-row transform blocks, whose signs and parities are
those of the global rows).  The factor of H_S and the controller then run
replicated on the summed values, so every rank takes the same decisions.

* `row_shards` cuts [0, n) into contiguous, block-aligned row ranges;
* `allreduce_sum` sums a tensor over the ranks of a torch.distributed group
  (NCCL for CUDA tensors, gloo for CPU tensors) in place, and is the identity
  when no group is initialised or it has one rank;
* `solve_sharded` runs ihs_solve_sharded on this rank's rows with
  `allreduce_sum` as the library's exchange step.
"""


def row_shards(n, parts, align=1):
    """Contiguous row ranges [(r0, r1)] covering [0, n) in `parts` blocks whose
    boundaries are multiples of `align` (a 1024-row FWHT block for the SRHT)."""
    if n < 1 or parts < 1 or align < 1:
        raise ValueError("need n >= 1, parts >= 1, align >= 1")
    units = -(-n // align)
    out = []
    for p in range(parts):
        u0, u1 = p * units // parts, (p + 1) * units // parts
        r0, r1 = min(n, u0 * align), min(n, u1 * align)
        if r1 > r0:
            out.append((r0, r1))
    return out


def _world(group=None):
    try:
        import torch.distributed as dist
    except ImportError:
        return None, 1
    if not (dist.is_available() and dist.is_initialized()):
        return None, 1
    return dist, dist.get_world_size(group)


def allreduce_sum(t, group=None):
    """Sum the tensor `t` over the ranks of `group` in place and return it;
    the identity with no initialised group or a single rank."""
    dist, world = _world(group)
    if world == 1:
        return t
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


class _DeviceBuffer:
    """A device buffer of the library, seen by torch without a copy."""

    def __init__(self, ptr, count, dtype):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8" if dtype == 1 else "<f4",
                                         "data": (int(ptr), False), "version": 2, "strides": None}


def make_allreduce(reduce_fn):
    """A C callback (ihs_allreduce_fn) that wraps the library's buffer in a torch
    tensor and calls reduce_fn(tensor) on the library's stream, which must sum it
    over the ranks in place.  Keep the returned object alive during the solve."""
    import torch

    from . import ihs

    @ihs.ALLREDUCE_FN
    def cb(user, buf, count, dtype, stream):
        try:
            t = torch.as_tensor(_DeviceBuffer(buf, count, dtype), device="cuda")
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                reduce_fn(t)
            return 0
        except Exception:   # reported to the caller as IHS_ECUDA
            return 1

    return cb


def solve_sharded(ctx, A_local, b_local, row0, n_total, nu, x, tol=0.0, group=None):
    """ihs_solve_sharded on this rank's rows [row0, row0 + len(A_local)) with the
    process group's all-reduce as the exchange; returns the report."""
    cb = make_allreduce(lambda t: allreduce_sum(t, group))
    return ctx.solve_sharded(A_local, b_local, row0, n_total, nu, x, cb, tol=tol)


__all__ = ["row_shards", "allreduce_sum", "make_allreduce", "solve_sharded"]
