"""Checkpoint and resume (nsk_save_checkpoint / nsk_load_checkpoint): stepping on from a
checkpoint written at a step boundary gives the same bits as never stopping (the low-storage
scheme's register holds nothing across steps: A_1 = 0), for FP64 and FP32 contexts and with the
1D sub-cell path's flags; the file's header holds what the format states; a context for another
mesh, a truncated file or a missing one are rejected with NSK_ERR_IO."""
import struct

import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs, nsk

pytestmark = pytest.mark.gpu

PRM = dict(T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3)


def _collision(precision, ne=(7, 6, 5)):
    s = nsk.Solver(3, ne, 3, [0, 0, 0], [1, 1, 1], 0, precision)
    s.set_params(**PRM)
    rv, rl, _ = O.maxwell(0.85)
    v = inputs.collision_velocity(40.0, 0.2, 1e-4, rv, rl)
    return s, inputs.head_on_collision(s.node_coords(), v, 0.2, rho_vap=rv, rho_liq=rl, kappa=1e-4)


@pytest.mark.parametrize("precision", [nsk.NSK_FP64, nsk.NSK_FP32_MIXED])
def test_resume_is_bit_exact(gpu, tmp_path, precision):
    s, U0 = _collision(precision)
    s.set_state(U0)
    dt = s.compute_dt(0.5)
    s.step(dt, 6)
    straight = s.get_state()
    s.set_state(U0)
    s.step(dt, 3)
    path = tmp_path / "state.ckpt"
    s.save_checkpoint(path, t=3 * dt, step=3)
    s.close()
    r, _ = _collision(precision)
    r.set_params(T=0.5, kappa=1.0, alpha=2.0, beta=1.0, mu=0.0)  # replaced by the file's parameters
    t, step = r.load_checkpoint(path)
    assert t == 3 * dt and step == 3
    r.step(dt, 3)
    assert np.array_equal(r.get_state(), straight)
    # header: magic, version, dim, N, node type, precision, model, flux, c dissipation, flags, nelem
    raw = path.read_bytes()
    assert raw[:8] == b"NSKCKPT\x00"
    ver, dim, N, nt, prec, model, flux, cd, nfl, nx, ny, nz = struct.unpack_from("<I11i", raw, 8)
    assert (ver, dim, N, nt, prec, nx, ny, nz) == (1, 3, 3, 0, precision, 7, 6, 5) and nfl == 0
    r.close()


def test_rejects_other_meshes_and_damaged_files(gpu, tmp_path):
    s, U0 = _collision(nsk.NSK_FP64)
    s.set_state(U0)
    path = tmp_path / "a.ckpt"
    s.save_checkpoint(path)
    other, _ = _collision(nsk.NSK_FP64, ne=(6, 6, 5))
    for target, p in ((other, path), (s, tmp_path / "missing.ckpt")):
        with pytest.raises(nsk.NskError) as ei:
            target.load_checkpoint(p)
        assert ei.value.code == nsk.NSK_ERR_IO
    short = tmp_path / "short.ckpt"
    short.write_bytes(path.read_bytes()[:-8])
    with pytest.raises(nsk.NskError) as ei:
        s.load_checkpoint(short)
    assert ei.value.code == nsk.NSK_ERR_IO
    other.close()
    s.close()


def test_subcell_flags_round_trip(gpu, tmp_path):
    def make():
        r = nsk.Solver(1, (40,), 3, [0.0], [1.0], 0, nsk.NSK_FP64)
        r.set_params(T=0.85, kappa=1e-6, alpha=100.0, beta=1e-3, mu=1e-3)
        r.set_flux(nsk.NSK_FLUX_HLLC)
        r.set_subcell(True, -6.0, -8.0)
        r.set_dirichlet((2.0, 0.0, 2.0), (0.1, 0.0, 0.1))
        return r

    r = make()
    r.set_state(inputs.riemann_1d(r.node_coords(), 2.0, 0.1, 0.5))
    r.step(1e-6, 5)
    flags, _ = r.subcell()
    assert flags.any()
    path = tmp_path / "fv.ckpt"
    r.save_checkpoint(path, t=5e-6, step=5)
    r.step(1e-6, 5)
    straight = r.get_state()
    q = make()
    q.load_checkpoint(path)
    assert np.array_equal(q.subcell()[0], flags)
    q.step(1e-6, 5)
    assert np.array_equal(q.get_state(), straight)
    q.close()
    r.close()
