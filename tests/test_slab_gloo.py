"""z-slab decomposition (paper_1301_3423_gb300/slab.py) on CPU ranks over gloo: each rank steps its
slab plus halo planes with the FP64 oracle as the stand-in step, exchanging only the population
planes that cross a slab face (|v_z| <= 6 for Q = 128, 3 for Q = 66; Eq. (rlb:disc), Sec. II.C).
The split run must equal the undivided oracle run bitwise, for periodic, copy-out and bounce-back
z ends."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1301_3423_gb300.slab import ZSlab  # noqa: E402
from paper_inputs import fields as gen  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (18, 4, 5)  # nz, ny, nx: 9 + 9 or 6 + 6 + 6 planes, each at least the reach
STEPS = 4


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def initial(order, bc):
    lat = oracle.read_lattice(order)
    nz, ny, nx = SHAPE
    n, T, u = gen.smooth_random_fields(SHAPE, seed=40 + order, vmax=0.4, sigma_lnT=0.15)
    o = oracle.OracleRLB(lat, nx, ny, nz, bc=bc, eta_over_s=0.1)
    o.init(n, T, u)
    return lat, o


def _rank_main(rank, world, port, order, bc, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lat, o = initial(order, bc)
    nz, ny, nx = SHAPE
    sl = ZSlab(lat.v, nz, rank, world, bc_z=bc[2])
    f = sl.scatter(o.f)
    ext = oracle.OracleRLB(lat, nx, ny, sl.nz_ext, bc=(bc[0], bc[1], sl.bc_ext()), eta_over_s=0.1)
    for _ in range(STEPS):
        sl.exchange(f)
        ext.set_populations(f)
        ext.step(1)
        f = ext.f.copy()
    np.save(os.path.join(out_dir, "rank%d.npy" % rank), f[:, sl.own()])
    dist.destroy_process_group()


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1), (0, 2, 2)])
@pytest.mark.parametrize("world", [2, 3])
def test_split_run_equals_the_undivided_run_bitwise(tmp_path, order, bc, world):
    lat, o = initial(order, bc)
    o.step(STEPS)
    mp.spawn(_rank_main, args=(world, free_port(), order, bc, str(tmp_path)), nprocs=world, join=True)
    parts = [np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world)]
    split = np.concatenate(parts, axis=1)
    assert split.shape == o.f.shape
    assert np.array_equal(split, o.f)


def test_exchanged_planes_are_the_crossing_populations():
    """Per face: sum over populations of max(v_z, 0) planes upward and max(-v_z, 0) downward."""
    lat = oracle.read_lattice(3)
    sl = ZSlab(lat.v, 64, 1, 4)
    up, down = sl.face_values(1, 1)
    assert up == int(np.sum(np.maximum(lat.v[:, 2], 0))) and down == int(np.sum(np.maximum(-lat.v[:, 2], 0)))
    assert sl.reach == 6 and sl.h_lo == sl.h_hi == 6 and sl.nzr == 16 and sl.z0 == 16
    with pytest.raises(ValueError):
        ZSlab(lat.v, 20, 0, 4)  # 5-plane slabs are shorter than the reach
    # ends without periodic wrap have no halo there
    end = ZSlab(lat.v, 64, 0, 4, bc_z=1)
    assert end.lower is None and end.h_lo == 0 and end.h_hi == 6
