"""Lattice geometry of Sec. 2.2-2.3 (oracle; test infrastructure only).

A periodic L0 x L1 x L2 x L3 lattice (x0 = time); sites in lexicographic order,
x0 slowest and x3 fastest.  Fields are numpy arrays whose first axis is the site.
"""
from __future__ import annotations

import numpy as np


class Lattice:
    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != 4 or min(self.dims) < 1:
            raise ValueError("need four positive extents")
        self.V = int(np.prod(self.dims))
        self.coords = np.indices(self.dims).reshape(4, -1).T.copy()  # [V, 4]
        # Sec. 6: x is even iff x0+x1+x2+x3 is even
        self.parity = self.coords.sum(axis=1) % 2

    def shift(self, f: np.ndarray, mu: int, sign: int) -> np.ndarray:
        """g(x) = f(x + sign * mu_hat), periodic (Sec. 2.2)."""
        rest = f.shape[1:]
        fr = f.reshape(self.dims + rest)
        g = np.roll(fr, -sign, axis=mu)
        return g.reshape(f.shape)

    def neighbour(self, mu: int, sign: int) -> np.ndarray:
        """Index of x + sign*mu_hat for every site x."""
        return self.shift(np.arange(self.V), mu, sign)


class Blocking:
    """A block decomposition of the lattice (Definition in Sec. 2.3) into equal blocks.

    Blocks are numbered lexicographically by their block coordinates; the block
    colour (red = 0, black = 1) is the parity of the block-coordinate sum.
    """

    def __init__(self, lat: Lattice, bdims):
        self.lat = lat
        self.bdims = tuple(int(b) for b in bdims)
        for L, b in zip(lat.dims, self.bdims):
            if b < 1 or L % b:
                raise ValueError("block extents must divide the lattice extents")
        self.nb_dims = tuple(L // b for L, b in zip(lat.dims, self.bdims))
        self.nblocks = int(np.prod(self.nb_dims))
        self.bvol = int(np.prod(self.bdims))
        bc = lat.coords // np.array(self.bdims)
        self.block_coords_of_site = bc
        self.block_of_site = np.ravel_multi_index(bc.T, self.nb_dims)
        self.block_coords = np.indices(self.nb_dims).reshape(4, -1).T.copy()
        self.colour = self.block_coords.sum(axis=1) % 2
        # sites of each block, lexicographic inside the block: [nblocks, bvol]
        order = np.argsort(self.block_of_site, kind="stable")
        self.sites = order.reshape(self.nblocks, self.bvol)

    def same_block(self, mu: int, sign: int) -> np.ndarray:
        """True where x and x + sign*mu lie in the same block (used for D_i = I^T D I)."""
        nb = self.lat.neighbour(mu, sign)
        return self.block_of_site[nb] == self.block_of_site
