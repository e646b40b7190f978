"""Full-size workloads in the launch configuration the benchmark times,
compared with the oracle on every pixel (the oracle finishes them in
seconds to a minute)."""
import numpy as np
import pytest

import oracle
from gpu_check import check_against_oracle
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_points_512_plain():
    m = inputs.points_512()
    check_against_oracle(m, 0)


@pytest.mark.parametrize("mode", [0, 1])
def test_discs_8192_both_modes(mode):
    m = inputs.discs_8192()
    check_against_oracle(m, mode, want_dist=False)


def test_blobs_512cube():
    m = inputs.blobs_512cube()
    check_against_oracle(m, 0, want_dist=False)
