"""Lattice geometry, block decomposition and active links (oracle).

Paper: Sec. 3 (block decomposition C, black/white checkerboard of blocks,
block-ordered labelling: black blocks first, then white blocks) and the
active-link rule (links with at most one endpoint on a block boundary).

Readings where the paper is silent:
  * canonical site index s = x0 + L0*(x1 + L1*(x2 + L2*x3)), axis 3 = time;
  * blocks tile [0, L) from the origin; block coordinate B_a = x_a // b_a;
    the number of blocks per direction is even (checkerboard), or 1, in
    which case a block spans that direction and keeps its wrap-around hops;
    block id = lexicographic in B; colour = (sum_a B_a) mod 2, 0 = black;
  * block ordering: black blocks in increasing block id, then white blocks,
    each block's sites in local lexicographic order;
  * active modes: "paper" applies the rule to the block itself; "inner6"
    applies it to the sub-block shrunk by one site on every side (a 6^4
    sub-block centred in an 8^4 block); "intra" takes every link with both
    ends in one block (needed for 2^4 blocks, where every site is a boundary
    site and the paper's set is empty); "auto" picks intra for blocks with an
    extent <= 2, inner6 for blocks with all extents >= 8, paper otherwise.
"""
import numpy as np

ACTIVE_MODES = ("paper", "inner6", "intra", "all")


def resolve_active_mode(block, mode="auto"):
    if mode != "auto":
        if mode not in ACTIVE_MODES:
            raise ValueError(f"unknown active mode {mode!r}")
        return mode
    if min(block) <= 2:
        return "intra"
    if min(block) >= 8:
        return "inner6"
    return "paper"


class Lattice:
    """Geometry of an L0 x L1 x L2 x L3 lattice with a block decomposition."""

    def __init__(self, dims, block=None, bc_time=-1, active_mode="auto"):
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != 4 or any(d < 2 or d % 2 for d in self.dims):
            raise ValueError("lattice extents must be four even numbers >= 2")
        self.block = tuple(int(b) for b in (block if block is not None else self.dims))
        self.bc_time = int(bc_time)
        L = np.array(self.dims)
        self.V = int(np.prod(L))
        s = np.arange(self.V)
        c = np.empty((self.V, 4), dtype=np.int64)
        c[:, 0] = s % L[0]
        c[:, 1] = (s // L[0]) % L[1]
        c[:, 2] = (s // (L[0] * L[1])) % L[2]
        c[:, 3] = s // (L[0] * L[1] * L[2])
        self.coords = c
        self.parity = c.sum(axis=1) % 2
        # nearest neighbours and the fermion boundary phase on time-wrapping hops
        self.fwd = np.empty((self.V, 4), dtype=np.int64)
        self.bwd = np.empty((self.V, 4), dtype=np.int64)
        self.sign_fwd = np.ones((self.V, 4))
        self.sign_bwd = np.ones((self.V, 4))
        for a in range(4):
            e = np.zeros(4, dtype=np.int64)
            e[a] = 1
            self.fwd[:, a] = self.index((c + e) % L)
            self.bwd[:, a] = self.index((c - e) % L)
        self.sign_fwd[c[:, 3] == L[3] - 1, 3] = self.bc_time
        self.sign_bwd[c[:, 3] == 0, 3] = self.bc_time
        self._init_blocks(active_mode)

    def index(self, c):
        L = self.dims
        return c[..., 0] + L[0] * (c[..., 1] + L[1] * (c[..., 2] + L[2] * c[..., 3]))

    # ------------------------------------------------------------------ blocks
    def _init_blocks(self, active_mode):
        b = np.array(self.block)
        L = np.array(self.dims)
        if np.any(L % b):
            raise ValueError("block extents must divide the lattice extents")
        nb = L // b
        if np.any((nb % 2) & (nb != 1)):
            raise ValueError("the number of blocks per direction must be even or 1 "
                             "(checkerboard colouring of the blocks)")
        self.nblock_dims = tuple(int(n) for n in nb)
        self.nblocks = int(np.prod(nb))
        self.block_sites = int(np.prod(b))
        B = self.coords // b
        self.block_coords = B
        self.block_id = B[:, 0] + nb[0] * (B[:, 1] + nb[1] * (B[:, 2] + nb[2] * B[:, 3]))
        self.colour = B.sum(axis=1) % 2
        loc = self.coords % b
        self.local = loc
        self.local_index = loc[:, 0] + b[0] * (loc[:, 1] + b[1] * (loc[:, 2] + b[2] * loc[:, 3]))
        # colour of every block, by block id
        bid = np.arange(self.nblocks)
        bc = np.stack([bid % nb[0], (bid // nb[0]) % nb[1],
                       (bid // (nb[0] * nb[1])) % nb[2], bid // (nb[0] * nb[1] * nb[2])], axis=1)
        self.block_colour = bc.sum(axis=1) % 2
        # block ordering: black blocks first (increasing id), then white blocks
        key = (self.colour * self.nblocks + self.block_id) * self.block_sites + self.local_index
        self.dd_order = np.argsort(key, kind="stable")      # dd position -> canonical site
        self.dd_pos = np.empty(self.V, dtype=np.int64)
        self.dd_pos[self.dd_order] = np.arange(self.V)      # canonical site -> dd position
        self.black_blocks = np.nonzero(self.block_colour == 0)[0]
        self.white_blocks = np.nonzero(self.block_colour == 1)[0]
        self.n_black_sites = int(np.sum(self.colour == 0))
        # boundary sites: a nearest neighbour lies in another block
        same = np.ones(self.V, dtype=bool)
        for a in range(4):
            same &= self.block_id[self.fwd[:, a]] == self.block_id
            same &= self.block_id[self.bwd[:, a]] == self.block_id
        self.on_boundary = ~same
        self.active_mode = resolve_active_mode(self.block, active_mode)
        self.active = self._active_links(self.active_mode)

    def _active_links(self, mode):
        """Boolean mask of shape (V, 4): link (s, a) is updated in the proposal."""
        act = np.zeros((self.V, 4), dtype=bool)
        if mode == "all":  # every link (pure-gauge updates of the whole lattice)
            act[:] = True
            return act
        if mode == "intra":
            for a in range(4):
                act[:, a] = self.block_id[self.fwd[:, a]] == self.block_id
            return act
        b = np.array(self.block)
        if mode == "paper":
            lo, hi = np.zeros(4, dtype=np.int64), b - 1
        else:  # inner6: the block shrunk by one site on each side
            if np.any(b < 4):
                raise ValueError("inner6 needs block extents >= 4")
            lo, hi = np.ones(4, dtype=np.int64), b - 2
        inside = np.all((self.local >= lo) & (self.local <= hi), axis=1)
        # a site of the region lies on its boundary when a neighbour is outside it
        region = np.where(inside, self.block_id, -1)
        on_bnd = np.zeros(self.V, dtype=bool)
        for a in range(4):
            on_bnd |= region[self.fwd[:, a]] != region
            on_bnd |= region[self.bwd[:, a]] != region
        on_bnd &= inside
        for a in range(4):
            y = self.fwd[:, a]
            both_in = inside & (region[y] == region)
            act[:, a] = both_in & ~(on_bnd & on_bnd[y])
        return act

    # -------------------------------------------------------------- helpers
    def block_sites_of(self, blk):
        """Canonical sites of block blk in local lexicographic order."""
        sites = np.nonzero(self.block_id == blk)[0]
        return sites[np.argsort(self.local_index[sites], kind="stable")]

    def black_sites(self):
        """Canonical sites of all black blocks, in block order."""
        return self.dd_order[: self.n_black_sites]

    def white_sites(self):
        return self.dd_order[self.n_black_sites:]

    def plaquettes(self):
        """All plaquettes as (site, a, b) with a < b; links (s,a),(s+a,b),(s+b,a),(s,b)."""
        out = []
        for a in range(4):
            for b in range(a + 1, 4):
                s = np.arange(self.V)
                out.append((s, a, b))
        return out
