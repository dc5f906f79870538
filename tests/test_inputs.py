"""The seeded input generators (inputs/): the properties the parity tests rely on."""
import numpy as np

import inputs


def test_start_columns_regenerate_alone():
    """Every column has its own stream: a subset equals the same columns of the whole block
    (the full-size parity test regenerates two of 512 columns for the oracle)."""
    full = inputs.start_columns("tiny", range(16))
    sub = inputs.start_columns("tiny", [3, 11])
    assert np.array_equal(sub, full[:, [3, 11]])
    again = inputs.start_columns("tiny", range(16))
    assert np.array_equal(again, full)
    assert not np.array_equal(full[:, 0], full[:, 1])


def test_systems_are_seeded():
    a, b = inputs.make_system("tiny"), inputs.make_system("tiny")
    for k in ("positions", "D", "dS"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]))
    c = inputs.make_system("tiny", seed=inputs.BASE_SEED + 1)
    assert not np.array_equal(np.asarray(a["D"]), np.asarray(c["D"]))
