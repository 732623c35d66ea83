"""Host side of surrogate persistence (train.write_surrogate / read_surrogate), CPU only:
the archive gives back exactly the arrays written, is written at the path given, and is
refused for a handle of other sizes or another prior, or when the arrays do not match the
descriptor."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2305_20053_gb300 import train


def _desc(**kw):
    d = dict(n=9, lattice_L=3, r_m=12, r_u=5, width=16, gamma=0.1, delta=1.0, m_mean=0.0)
    d.update(kw)
    return SimpleNamespace(**d)


def _arrays(desc, seed=3):
    rng = np.random.default_rng(seed)
    n, r_u = desc.n, desc.r_u
    params = rng.standard_normal(123).astype(np.float32)
    scale = rng.uniform(0.01, 0.1, r_u).astype(np.float32)
    phi = rng.standard_normal((r_u, n, n))
    phi[:, 0, :] = phi[:, -1, :] = phi[:, :, 0] = phi[:, :, -1] = 0.0
    ubar = rng.standard_normal((n, n))
    return params, scale, phi, ubar


def test_round_trip_is_exact(tmp_path):
    desc = _desc()
    params, scale, phi, ubar = _arrays(desc)
    path = tmp_path / "net.surrogate"
    train.write_surrogate(str(path), desc, params, scale, phi, ubar)
    assert path.exists() and not (tmp_path / "net.surrogate.npz").exists()
    a = train.read_surrogate(str(path), _desc())
    assert a["params"].dtype == np.float32 and np.array_equal(a["params"], params)
    assert a["out_scale"].dtype == np.float32 and np.array_equal(a["out_scale"], scale)
    assert a["phi"].dtype == np.float64 and np.array_equal(a["phi"], phi)
    assert a["ubar"].dtype == np.float64 and np.array_equal(a["ubar"], ubar)


@pytest.mark.parametrize("field,value", [("n", 17), ("r_m", 10), ("width", 24), ("gamma", 0.2), ("m_mean", -1.0)])
def test_refused_for_other_sizes_or_prior(tmp_path, field, value):
    desc = _desc()
    path = tmp_path / "net.npz"
    train.write_surrogate(str(path), desc, *_arrays(desc))
    with pytest.raises(ValueError, match=field):
        train.read_surrogate(str(path), _desc(**{field: value}))


def test_arrays_must_match_descriptor(tmp_path):
    desc = _desc()
    params, scale, phi, ubar = _arrays(desc)
    with pytest.raises(ValueError):
        train.write_surrogate(str(tmp_path / "a.npz"), desc, params, scale[:-1], phi, ubar)
    with pytest.raises(ValueError):
        train.write_surrogate(str(tmp_path / "b.npz"), desc, params, scale, phi[:, :-1], ubar)
    with pytest.raises(ValueError):
        train.write_surrogate(str(tmp_path / "c.npz"), _desc(r_u=4), params, scale, phi, ubar)
