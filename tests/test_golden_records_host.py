"""The stored oracle records are well formed and their sample positions are the ones their
committed generators draw (no GPU)."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_turbulence64_record_matches_its_generator_positions():
    spec = importlib.util.spec_from_file_location("make_turbulence64", os.path.join(HERE, "golden",
                                                                                    "make_turbulence64.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    pos = gen.sample_positions()
    rows = []
    head = {}
    with open(os.path.join(HERE, "golden", "turbulence64_d3q27_fp64.txt")) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("maxabs", "mass", "kinetic_energy", "momentum"):
                head[parts[0]] = [float(v) for v in parts[1:]]
            else:
                rows.append([int(v) for v in parts[:4]] + [float(parts[4])])
    rows = np.array(rows)
    assert rows.shape == (gen.SAMPLES, 5)
    np.testing.assert_array_equal(rows[:, :4].astype(int), pos)
    # a physical state: PDFs positive and below max |f|, mass = cells (rho = 1 start) to rounding
    assert np.all(rows[:, 4] > 0) and np.all(rows[:, 4] <= head["maxabs"][0])
    assert abs(head["mass"][0] / gen.N ** 3 - 1) < 1e-12


def test_porous_minibed_record_matches_its_generator_positions():
    spec = importlib.util.spec_from_file_location("make_porous_minibed",
                                                  os.path.join(HERE, "golden", "make_porous_minibed.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    _, shape, flags = gen.geometry()
    pos = gen.sample_positions(flags)
    rows, head = [], {}
    with open(os.path.join(HERE, "golden", "porous_minibed_fp64.txt")) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("maxabs", "mass", "momentum"):
                head[parts[0]] = [float(v) for v in parts[1:]]
            else:
                rows.append([int(v) for v in parts[:4]] + [float(parts[4])])
    rows = np.array(rows)
    assert rows.shape == (gen.SAMPLES, 5)
    np.testing.assert_array_equal(rows[:, :4].astype(int), pos)
    assert np.all(flags[pos[:, 1], pos[:, 2], pos[:, 3]] == 0)  # fluid cells only
    assert np.all(rows[:, 4] > 0) and np.all(rows[:, 4] <= head["maxabs"][0])
    # the inlet pushes ~470 mass units per step into a bed that is still building the pressure
    # that drives the flow through it: after 1,000 steps the mean density is ~1.2
    fluid = int((flags == 0).sum())
    assert 1.0 < head["mass"][0] / fluid < 1.5
    assert head["momentum"][0] > 0  # the flow runs from the inlet to the outlet


def test_channel_column_record_is_the_oracle_column():
    """The column the benchmark states its variants' errors against is the oracle's own run (the
    generator's column() recomputed here), bit for bit, for TRT and MRT."""
    spec = importlib.util.spec_from_file_location("make_channel_column",
                                                  os.path.join(HERE, "golden", "make_channel_column.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    import oracle
    rec = gen.read()
    assert set(rec) == {"trt", "mrt"}
    for name, coll in (("trt", oracle.TRT), ("mrt", oracle.MRT)):
        assert rec[name].shape == (19, gen.H)
        np.testing.assert_array_equal(rec[name], gen.column(coll))
    # the flow is developed but far from steady: centre-line u_x ~ F t
    c, _, _ = oracle.lattice(19)
    f = rec["trt"]
    ux = c[:, 0] @ f / f.sum(0)
    assert 1.5e-3 < ux[gen.H // 2] <= (gen.STEPS + 0.5) * 1e-6  # post-collision: + F/2
