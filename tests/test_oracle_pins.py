"""The CPU oracle against its pins (no GPU)."""
import pytest

from paper_2511_16298_gb300 import synth
from tests import oracle_pins as P


def test_golden_hand_frame(oracle):
    P.check_golden(oracle)


def test_count_and_duplicate_brute_force(oracle):
    P.check_count_and_duplicate_bruteforce(oracle, seeds=range(120))


def test_special_cases(oracle):
    P.check_special_cases(oracle)


def test_validity(oracle):
    P.check_validity(oracle)


def test_scan(oracle):
    P.check_scan(oracle)


def test_sort(oracle):
    P.check_sort(oracle)


def test_float_bit_order():
    P.check_float_order()


@pytest.mark.parametrize("make", [
    lambda: synth.frame_small(0),
    lambda: synth.frame_small(5, n=3000, width=200, height=120),
    lambda: synth.frame_random(1, 5000, 333, 177, depth_ties=0.3),
    lambda: synth.frame_random(2, 2000, 16, 16),
    lambda: synth.frame_large(0, n=40_000, width=640, height=360),
])
def test_frame_invariants(oracle, make):
    P.check_frame_invariants(oracle, [make()])


def test_preprocess_pins(oracle):
    """Projection and footprint (Sec. II-A "Preprocessing"; Tables I and IV)."""
    P.check_preprocess(oracle)


def test_render_pins(oracle):
    """Front-to-back blending (Sec. II-A "Rendering"; Sec. IV-C)."""
    P.check_render(oracle)


def test_normalized_pins(oracle):
    """The 32-bit tile/depth key (Sec. IV-B)."""
    P.check_normalized(oracle)
