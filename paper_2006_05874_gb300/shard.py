"""Row sharding of the path on a single GPU.

The method shards by rows of A: every per-row quantity stays local and the
gradient needs one sum of d floats (and of ||A x||^2) over the shards,

    grad f(x) = sum_p A_p^T (A_p x - b_p) + nu^2 x,

which `ihs_grad` computes per shard when nu^2 x is added on shard 0 only (the
sketches have the same form: the SRHT and Gaussian kernels already sum per
row-group partials in a fixed order).  With one GPU per process the collective
is the identity: `allreduce_sum` is the seam a multi-GPU build would fill, and
on one GPU it returns its argument."""


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


def allreduce_sum(buf, world_size=1):
    """The sum over ranks of `buf`; with one rank (every process of this
    library drives one GPU) the identity."""
    if world_size != 1:
        raise NotImplementedError("one GPU per process: the collective is the identity")
    return buf
