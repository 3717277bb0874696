"""The decode kernels divide 64-bit point indices by divisors fixed for a launch
with a multiply-high by m = floor((2^64 - 1) / d) and at most two remainder
corrections (division by invariant integers, Granlund and Montgomery 1994).
This checks that claim in exact integer arithmetic, the same steps as the
device function: the estimate is q, q - 1 or q - 2 for every numerator below
2^64, and the corrected quotient equals floor division.
"""
import random

import pytest

M64 = (1 << 64) - 1


def fdiv_steps(num, d):
    m = M64 // d
    q = (num * m) >> 64
    r = (num - q * d) & M64
    fixes = 0
    for _ in range(2):
        if r >= d:
            q += 1
            r -= d
            fixes += 1
    return q, r, fixes


@pytest.mark.parametrize("seed", range(4))
def test_fastdiv_equals_floor_division(seed):
    rng = random.Random(seed)
    divisors = [1, 2, 3, 7, 255, 256, 257, 511, 4095, 2 * 511, 2 * 1023, (1 << 32) - 1, 1 << 32,
                (1 << 63) - 1, 1 << 63, M64]
    divisors += [rng.randrange(1, 1 << rng.randrange(1, 65)) for _ in range(200)]
    for d in divisors:
        nums = [0, 1, d - 1, d, d + 1, M64, M64 - 1, M64 - d, (1 << 62), (1 << 56) + 12345]
        nums += [rng.randrange(0, 1 << rng.randrange(1, 65)) for _ in range(50)]
        for num in nums:
            num &= M64
            q, r, fixes = fdiv_steps(num, d)
            assert q == num // d and r == num % d and fixes <= 2, (num, d, q, fixes)


def test_grid_coordinate_formula():
    # the voxel -> fixed-point map of decode_grid: floor((2^25 j + n - 1) / (2 (n - 1)))
    # is round-half-up of j / (n - 1) * 2^24, exact through the fast division
    for n in (2, 3, 64, 258, 514, 4097):
        D = 2 * (n - 1)
        for j in range(0, n, max(1, n // 97)):
            q, _, _ = fdiv_steps((j << 25) + n - 1, D)
            assert q == ((j << 25) + n - 1) // D
            assert q == (2 * j * (1 << 24) + (n - 1)) // (2 * (n - 1))
    assert fdiv_steps(((4096) << 25) + 4096, 2 * 4096)[0] == 1 << 24
