"""bench.py's host-side bookkeeping without a GPU: the roofline's algorithmic unit counts for
the table, ACA and transfer kernels, the exclusion of library calls from the dominant-kernel
pick, and the source-hash check that voids stale DRAM-traffic figures."""
import hashlib
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PK = {"sm_max_mhz": 2070.0, "bf16_tflops": 1888.0}


def _info(**levels):
    info = {k: [0] * 22 for k in ("mode", "r1", "L", "nQ", "n_adm", "n_trans", "pw_prec", "pw_recurrences",
                                  "tune_tc", "aca_rank", "aca_terms", "aca_pair_terms", "src_points",
                                  "tgt_points")}
    info["cancel"] = [0.0] * 22
    info["p2p_pairs"] = 0
    for key, vals in levels.items():
        for l, v in vals.items():
            info[key][l] = v
    return info


def test_library_calls_are_listed_but_not_ranked():
    prof = {"cufftExecC2C (library)": (4, 40.0), "k_lag_aca": (5, 2.0)}
    info = _info(mode={2: 1}, r1={2: 4}, n_trans={2: 316}, aca_rank={2: 20}, aca_terms={2: 5000})
    out = bench.roofline(prof, info, 1, 2070.0, PK, "measured", "laplace_sphere_20k")
    assert out["kernel"] == "k_lag_aca"


def test_aca_units_count_every_term_over_the_whole_residual():
    r = 4 ** 3
    info = _info(mode={2: 1, 3: 1}, r1={2: 4, 3: 4}, n_trans={2: 316, 3: 664}, aca_rank={2: 20, 3: 21},
                 aca_terms={2: 5000, 3: 11000})
    out = bench.roofline({"k_lag_aca": (2, 1.0)}, info, 1, 2070.0, PK, "measured", "laplace_sphere_20k")
    units = 3.0 * r * r * (5000 + 316 + 11000 + 664)
    assert out["units_per_step"] == pytest.approx(units)
    assert out["achieved"] == pytest.approx(units / 1e-3 / 1e12)
    assert out["frac"] == pytest.approx(out["achieved"] / 1.25)


def test_transfer_units_use_the_aca_ranks_per_pair_on_aca_levels():
    info = _info(mode={2: 1, 3: 1}, r1={2: 4, 3: 4}, n_adm={2: 1000, 3: 5000}, tune_tc={2: 1, 3: 1},
                 aca_rank={3: 20}, aca_pair_terms={3: 80000})
    out = bench.roofline({"(k_lag_gemm_tc<KT, NR, NO>)": (3, 1.0)}, info, 1, 2070.0, PK, "measured",
                         "laplace_sphere_20k")
    assert out["units_per_step"] == pytest.approx(2.0 * 64 * 64 * 1000 + 4.0 * 64 * 80000)


def test_gegenbauer_table_units_follow_each_levels_table_kernel():
    # levels 2-4 FP32 and well conditioned (FP32 table), level 5 compensated (double-float table)
    info = _info(mode={2: 2, 3: 2, 4: 2, 5: 2}, L={2: 100, 3: 50, 4: 30, 5: 20},
                 pw_prec={2: 1, 3: 1, 4: 1, 5: 2}, pw_recurrences={2: 10, 3: 20, 4: 30, 5: 40})
    info["cancel"][2:6] = [10.0, 20.0, 30.0, 900.0]
    f32 = bench.roofline({"k_pw_table_f32": (3, 1.0)}, info, 1, 2070.0, PK, "measured", "helmholtz_sphere_1M")
    dd = bench.roofline({"k_pw_table<float2>": (1, 1.0)}, info, 1, 2070.0, PK, "measured", "helmholtz_sphere_1M")
    assert f32["units_per_step"] == pytest.approx(19.0 * (10 * 100 + 20 * 50 + 30 * 30))
    assert dd["units_per_step"] == pytest.approx(72.0 * 40 * 20)


def test_tensor_core_transform_units_count_each_levels_points_directions_and_columns():
    # levels 2, 3 FP32, level 4 compensated, level 5 double-float; 64 right-hand sides
    info = _info(mode={2: 2, 3: 2, 4: 2, 5: 2}, nQ={2: 6844, 3: 2380, 4: 924, 5: 480},
                 pw_prec={2: 1, 3: 1, 4: 2, 5: 4}, src_points={2: 200000, 3: 199000, 4: 198000, 5: 190000},
                 tgt_points={2: 150000, 3: 149000, 4: 148000, 5: 140000}, n_adm={2: 2504, 3: 12960, 5: 184896})
    fwd = bench.roofline({"k_pw_forward_tc<f32>": (2, 4.0)}, info, 1, 2070.0, PK, "measured", "cube", nrhs=64)
    assert fwd["bound"] == "tensor"
    assert fwd["units_per_step"] == pytest.approx(8.0 * 64 * (200000 * 3422 + 199000 * 1190))
    fwc = bench.roofline({"k_pw_forward_tc<f32c>": (1, 1.0)}, info, 1, 2070.0, PK, "measured", "cube", nrhs=64)
    assert fwc["units_per_step"] == pytest.approx(8.0 * 64 * 198000 * 462)
    bwd = bench.roofline({"k_pw_backward_tc<f32>": (2, 4.0)}, info, 1, 2070.0, PK, "measured", "cube", nrhs=64)
    assert bwd["units_per_step"] == pytest.approx(8.0 * 64 * (150000 * 3422 + 149000 * 1190))
    tr = bench.roofline({"k_pw_transfer<f32x2>": (1, 17.0)}, info, 1, 2070.0, PK, "measured", "cube", nrhs=64)
    assert tr["bound"] == "alu" and tr["units_per_step"] == pytest.approx(72.0 * 64 * 184896 * 480)
    bdd = bench.roofline({"k_pw_backward_mr<f32x2>": (1, 16.0)}, info, 1, 2070.0, PK, "measured", "cube", nrhs=64)
    assert bdd["units_per_step"] == pytest.approx(72.0 * 64 * 140000 * 240)


def test_traffic_figures_are_void_once_the_kernel_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "paper_1909_05600_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("kernel v1\n")
    h = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment\nk_x<W> wl_small 12.5 pair k.cu %s\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    tr = bench.measured_traffic("k_x<W>")
    assert tr["bytes_per_unit"] == 12.5 and tr["captured_on"] == "wl_small"
    assert bench.measured_traffic("k_y") is None
    (src / "k.cu").write_text("kernel v2\n")
    assert bench.measured_traffic("k_x<W>") is None


def test_roofline_traffic_scales_the_per_unit_figure_to_the_launch(tmp_path, monkeypatch):
    src = tmp_path / "paper_1909_05600_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "nearfield.cu").write_text("v\n")
    h = hashlib.sha256(b"v\n").hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text("k_p2p_lap<4> small 0.5 pair nearfield.cu %s\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    info = _info()
    info["p2p_pairs"] = 1000
    rl = bench.roofline({"k_p2p_lap<4>": (2, 4.0)}, info, 2, 2070.0, PK, "measured", "laplace_clustered")
    assert rl["units_per_step"] == 1000.0
    assert rl["traffic"] == pytest.approx(0.5 * 1000.0 / 1.0)
