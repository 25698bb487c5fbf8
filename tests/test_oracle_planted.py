"""Mutation testing of the oracle's pins.

The oracle is rebuilt with one known, plausible mistake planted
(-DORC_PLANT=k: a flipped sign, a transposed operand, a wrong constant, a
dropped term, an off-by-one; 1 .. 12, 17, 18 in oracle.c, 13 .. 16 in oracle_mlp.c) and the pins are run against it: for every
planted mistake at least one pin must fail. This is what makes the pins
evidence that the unplanted oracle computes what the paper defines.
"""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O

import test_oracle_dft as TD
import test_oracle_mlp as TM
import test_oracle_sphere as TS
import test_oracle_tree as TT
import test_oracle_truncated as TR

HERE = os.path.dirname(os.path.abspath(O.__file__))

# planted mistake -> the pins that should notice it (at least one must fail)
PLANTS = {
    1: ("n - 1 with the wrong sign", [TD.test_symmetric_pair_closed_form, TD.test_fp64_against_long_double]),
    2: ("v multiplied by l instead of m", [TD.test_two_component_modulus_closed_form]),
    3: ("R_x(+dec) instead of R_x(-dec)",
        [lambda: TS.test_rotation_maps_phase_centre_east_north(np.pi, np.radians(45))]),
    4: ("off-by-one in the equatorial y index", [TS.test_golden_nested_points,
                                                 lambda: TS.test_round_trip_every_pixel(2)]),
    5: ("longitude scaled by pi instead of pi/2", [TS.test_golden_nested_points, TS.test_equal_area_monte_carlo]),
    6: ("Eq. 9 average with 1/2 instead of 1/4", [lambda: TT.test_eq17_equals_eq16(8),
                                                  lambda: TT.test_brute_force_dense_grid(5)]),
    7: ("Eq. 10 second row with a wrong sign", [lambda: TT.test_eq17_equals_eq16(8),
                                                lambda: TT.test_brute_force_dense_grid(5)]),
    8: ("Eq. 17 level-1 term without A_1", [lambda: TT.test_eq17_equals_eq16(8)]),
    9: ("merged flux overwritten instead of summed", [TT.test_bfs_structure_invariants]),
    10: ("equatorial ring height doubled", [lambda: TS.test_round_trip_every_pixel(2), TS.test_base_pixel_centres]),
    11: ("s_w - 1 with the wrong sign", [lambda: TT.test_eq16_is_direct_sum_at_pixel_centres(10),
                                        TS.test_pixel_dir_uvw_of_phase_centre_pixel]),
    12: ("plane-wave sigma^0 with a wrong sign", [lambda: TT.test_eq17_equals_eq16(8)]),
    13: ("pixel response with the sub-pixel offsets reversed", [TM.test_pixel_response_is_the_direct_sum_over_subpixel_centres]),
    14: ("pixel response normalised by 4^(D-1)", [TM.test_pixel_response_at_zero_baseline_is_one]),
    15: ("SiLU derivative without its z (1 - s) term", [TM.test_mlp_gradient_matches_finite_differences]),
    16: ("second weight matrix transposed in the forward pass", [TM.test_mlp_forward_closed_form,
                                                                  TM.test_mlp_gradient_matches_finite_differences]),
    17: ("truncated tree weighted by lambda instead of the pixel's flux A_jt lambda",
         [TR.test_truncated_at_level_J_is_eq16, lambda: TR.test_fully_populated_phase_centre_pixel_is_eq12("level")]),
    18: ("truncated tree with the pixel response conjugated",
         [lambda: TR.test_fully_populated_phase_centre_pixel_is_eq12("level"),
          lambda: TR.test_fully_populated_phase_centre_pixel_is_eq12("pixel")]),
}


def _build_planted(k, outdir):
    srcs = [os.path.join(HERE, s) for s in ("oracle.c", "oracle_mlp.c")]
    lib = os.path.join(outdir, "liboracle_plant%d.so" % k)
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
                           "-DORC_PLANT=%d" % k, "-o", lib] + srcs + ["-lm"])
    L = C.CDLL(lib)
    O._declare(L)
    return L


@pytest.fixture(scope="module")
def plant_dir():
    with tempfile.TemporaryDirectory() as d:
        yield d


@pytest.mark.parametrize("k", sorted(PLANTS))
def test_every_planted_mistake_fails_a_pin(k, plant_dir, monkeypatch):
    what, pins = PLANTS[k]
    monkeypatch.setattr(O, "_lib", _build_planted(k, plant_dir))
    failed = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError) as e:
            failed.append(e)
    assert failed, "planted mistake %d (%s) passed every pin" % (k, what)


def test_unplanted_build_passes_the_same_pins(plant_dir, monkeypatch):
    monkeypatch.setattr(O, "_lib", _build_planted(0, plant_dir))
    for _, pins in PLANTS.values():
        for pin in pins:
            pin()
