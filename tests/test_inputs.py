"""Seeded input generators (no GPU): the splitmix64 stream and the ragged
ensemble draws."""
import ptt_inputs as I
from oracle import ptt2d as O


def test_splitmix64_first_outputs_of_seed_zero():
    # the published first outputs of splitmix64 started from state 0
    assert I.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert I.splitmix64(0, 1) == 0x6E789E6AA1B965F4


def test_unit_draws_agree_with_the_oracle_generator():
    # both sides implement the generator; the uniform [-1, 1) of the oracle is
    # 2 u - 1 of the same 53-bit draw
    for seed in (0, 3, 12345):
        for k in (0, 1, 7, 100):
            assert O.splitmix_uniform(seed, k) == 2.0 * I.splitmix_unit(seed, k) - 1.0


def test_ensemble_draws_cover_the_ranges():
    m = I.ensemble_members()
    nx = {a for a, _, _, _ in m}
    ny = {b for _, b, _, _ in m}
    wi = [w for _, _, w, _ in m]
    assert len(m) == 64 and [s for *_, s in m] == list(range(64))
    assert nx <= set(I.ENSEMBLE_NX) and ny <= set(I.ENSEMBLE_NY)
    assert len(nx) >= 8 and len(ny) >= 5
    assert 50.0 <= min(wi) and max(wi) <= 200.0
    assert all(n % 32 == 0 and 64 <= n <= 512 for n in nx)
    # the full sets of the configuration: every multiple of 32, Ny up to 257
    # with 225 (ny - 1 = 2^5 7), and the draws reach the radix-7/11/13 sizes
    assert I.ENSEMBLE_NX == tuple(range(64, 513, 32))
    assert I.ENSEMBLE_NY == (65, 97, 129, 161, 193, 225, 257)
    assert nx & {224, 352, 416, 448} and 225 in ny
