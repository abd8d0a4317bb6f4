"""One map over several ranks (one process per GPU).

Rays are independent (the ray-shooting loop of Sec. 2.4 has no coupling
between rays), so the lattice rows are cut into strips of whole level-1 cell
rows (whole 64-row tiles for the brute force), each rank shoots its strip
through irs_make_map_rows into its own count map, and the partial maps are
summed: one reduction of npix_x * npix_y uint32 values is the only exchange.
Every rank holds all lenses and builds the whole far field (it is ~15 % of a
map at the paper-mid workload); the cell rows are dealt as evenly as they go.
"""
from . import irs

BRUTE_TILE_ROWS = 64  # lattice rows of one brute-force tile


def strip_rows(n_rows, world, rank, align=1):
    """Lattice rows [r0, r1) of `rank`'s strip: blocks of `align` rows dealt
    so that strip sizes differ by at most one block.  Strips tile [0, n_rows)."""
    if world < 1 or not 0 <= rank < world or align < 1 or n_rows < 0:
        raise ValueError("bad strip request")
    nblk = -(-n_rows // align)
    b0, b1 = rank * nblk // world, (rank + 1) * nblk // world
    return min(b0 * align, n_rows), min(b1 * align, n_rows)


def row_align(plan):
    """Rows per strip block: one level-1 cell row, or one brute-force tile row."""
    k = int(plan.info.rays_per_cell_y)
    return k if k > 0 else BRUTE_TILE_ROWS


def sum_maps(counts, group=None):
    """Sum the ranks' partial uint32 count maps in place on every rank.  The
    reduction runs on the int32 view (two's-complement addition is the same
    bit pattern as uint32 addition mod 2^32)."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(counts.view(torch.int32), op=dist.ReduceOp.SUM, group=group)


def make_map_sharded(plan, lens_xy, mass, counts, world, rank, mag=None, group=None, stream=None):
    """This rank's strip of the map, then the sum over ranks (and Mag if asked)."""
    r0, r1 = strip_rows(int(plan.info.n_rays_y), world, rank, row_align(plan))
    counts.zero_()
    if r1 > r0:
        irs.irs_make_map_rows(plan.handle, lens_xy, mass, r0, r1, counts, stream)
    if world > 1:
        sum_maps(counts, group)
    if mag is not None:
        irs.irs_magnify(plan.handle, counts, mag, stream)
    return r0, r1
