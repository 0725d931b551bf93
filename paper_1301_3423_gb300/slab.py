"""z-slab decomposition of one lattice over ranks, with the halo exchange of one time step.

The pull of Eq. (rlb:disc) moves population i by the integer vector v_i, and |v_i,z| is at most
VMAX_Z (6 for the third-order model, R^2 = 41; 3 for the second-order one, R^2 = 9; Sec. II.C and
App. A).  Splitting the lattice into contiguous z ranges ("slabs") therefore needs, before each
step, only the populations that cross a slab face: population i with v_i,z = d > 0 at the first d
planes of a slab pulls from the last d planes of the slab below, and one with d < 0 at the last |d|
planes from the first |d| planes of the slab above.  Each rank holds its slab plus halo planes
(VMAX_Z on each side that has a neighbour), sends exactly those population planes to its two
neighbours once per step (point-to-point, torch.distributed: gloo or NCCL), and then steps the
extended lattice; only its own planes are kept, the halo planes are refilled by the next exchange.
Per face and step that is sum_i max(v_i,z, 0) population planes of nx * ny values (about 200 planes
for Q = 128), against Q planes per slab plane of streaming work.

The global z boundary stays where it is: with a periodic z the first and last ranks are neighbours;
with copy-out or bounce-back ends the ranks at the ends have no halo there and their extended
lattice carries the same boundary (the opposite end of their extended lattice lies in a halo, and
only halo planes can see it).  Every interior cell pulls the same values as in the undivided run,
so a step that is exact per cell gives the undivided result bitwise.

This module is the host side of the decomposition: partition, packing and exchange.  The step
itself is the caller's (the library's step on each rank's own device).
"""
import numpy as np


class ZSlab:
    """One rank's part of an nx x ny x nz lattice split along z over `world` ranks.

    v: (q, 3) integer velocities; bc_z: 0 periodic, 1 copy-out, 2 bounce-back (both ends)."""

    def __init__(self, v, nz, rank, world, bc_z=0):
        v = np.asarray(v, dtype=np.int64)
        self.q = len(v)
        self.vz = v[:, 2]
        self.reach = int(np.max(np.abs(self.vz)))
        self.nz, self.rank, self.world, self.bc_z = int(nz), int(rank), int(world), int(bc_z)
        base, extra = divmod(self.nz, self.world)
        sizes = [base + (1 if r < extra else 0) for r in range(self.world)]
        if min(sizes) < self.reach:
            raise ValueError("every slab needs at least %d planes (the stencil reach); %d planes over %d ranks "
                             "give %d" % (self.reach, self.nz, self.world, min(sizes)))
        self.z0 = sum(sizes[:self.rank])
        self.nzr = sizes[self.rank]
        periodic = self.bc_z == 0
        self.lower = (self.rank - 1) % self.world if (periodic or self.rank > 0) else None
        self.upper = (self.rank + 1) % self.world if (periodic or self.rank < self.world - 1) else None
        self.h_lo = self.reach if self.lower is not None else 0
        self.h_hi = self.reach if self.upper is not None else 0
        # populations that cross each face, with their depth in planes
        self.up = [(i, int(d)) for i, d in enumerate(self.vz) if d > 0]      # my top d planes -> upper's bottom halo
        self.down = [(i, int(-d)) for i, d in enumerate(self.vz) if d < 0]   # my bottom |d| planes -> lower's top halo

    @property
    def nz_ext(self):
        return self.h_lo + self.nzr + self.h_hi

    def bc_ext(self):
        """z boundary of the extended lattice: the global one at a global end; at a halo end any
        boundary gives the same interior (copy-out is used)."""
        return 1 if self.bc_z == 0 else self.bc_z

    def own(self):
        """Slice of the extended lattice's z axis holding this rank's planes."""
        return slice(self.h_lo, self.h_lo + self.nzr)

    def scatter(self, f_global):
        """This rank's extended array (q, nz_ext, ny, nx) from the whole lattice's populations (halo
        planes zero until the first exchange)."""
        q, nz, ny, nx = f_global.shape
        out = np.zeros((q, self.nz_ext, ny, nx), dtype=f_global.dtype)
        out[:, self.own()] = f_global[:, self.z0:self.z0 + self.nzr]
        return out

    def face_values(self, nx, ny):
        """Values per exchanged buffer: (to the upper neighbour, to the lower neighbour)."""
        return (sum(d for _, d in self.up) * nx * ny, sum(d for _, d in self.down) * nx * ny)

    def pack_up(self, f_ext):
        top = self.h_lo + self.nzr
        return np.concatenate([f_ext[i, top - d:top].ravel() for i, d in self.up])

    def pack_down(self, f_ext):
        bot = self.h_lo
        return np.concatenate([f_ext[i, bot:bot + d].ravel() for i, d in self.down])

    def unpack_from_lower(self, f_ext, buf):
        """The lower neighbour's top planes of the upward populations into my bottom halo."""
        ny, nx = f_ext.shape[2:]
        k = 0
        for i, d in self.up:
            n = d * ny * nx
            f_ext[i, self.h_lo - d:self.h_lo] = buf[k:k + n].reshape(d, ny, nx)
            k += n

    def unpack_from_upper(self, f_ext, buf):
        """The upper neighbour's bottom planes of the downward populations into my top halo."""
        ny, nx = f_ext.shape[2:]
        top = self.h_lo + self.nzr
        k = 0
        for i, d in self.down:
            n = d * ny * nx
            f_ext[i, top:top + d] = buf[k:k + n].reshape(d, ny, nx)
            k += n

    def exchange(self, f_ext):
        """Fill the halo planes of f_ext (numpy, updated in place) from the neighbours over the
        default torch.distributed process group (one send and one receive per face, tags 0 for
        upward and 1 for downward traffic).  With a single periodic rank the faces are its own."""
        import torch
        import torch.distributed as dist

        ny, nx = f_ext.shape[2:]
        n_up, n_down = self.face_values(nx, ny)
        to_up = torch.from_numpy(self.pack_up(f_ext)) if self.upper is not None else None
        to_down = torch.from_numpy(self.pack_down(f_ext)) if self.lower is not None else None
        if self.world == 1:
            if self.lower is not None:
                self.unpack_from_lower(f_ext, to_up.numpy())
                self.unpack_from_upper(f_ext, to_down.numpy())
            return
        from_lower = torch.empty(n_up, dtype=to_up.dtype if to_up is not None else torch.float64) \
            if self.lower is not None else None
        from_upper = torch.empty(n_down, dtype=from_lower.dtype if from_lower is not None else torch.float64) \
            if self.upper is not None else None
        ops = []
        if self.upper is not None:
            ops.append(dist.P2POp(dist.isend, to_up, self.upper, tag=0))
            ops.append(dist.P2POp(dist.irecv, from_upper, self.upper, tag=1))
        if self.lower is not None:
            ops.append(dist.P2POp(dist.isend, to_down, self.lower, tag=1))
            ops.append(dist.P2POp(dist.irecv, from_lower, self.lower, tag=0))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        if self.lower is not None:
            self.unpack_from_lower(f_ext, from_lower.numpy())
        if self.upper is not None:
            self.unpack_from_upper(f_ext, from_upper.numpy())
