"""The mixed-precision warp path takes the RKC stage count in FP32:
s = floor(1 + sqrtf(1 + (float)(1.54 h sigma))) (Section 2.3's stage rule).
IEEE FP32 addition and square root are correctly rounded on the GPU and in
numpy alike, so numpy reproduces the device's FP32 arithmetic here. The test
shows what the design relies on: the FP32 count equals the FP64 count except
where 1 + sqrt(1 + 1.54 h sigma) lies within FP32 rounding of an integer, and
such steps are rare over the range of h sigma the 250-stage cap allows."""
import numpy as np

S_MAX = 250


def stage_counts(z64):
    s64 = np.floor(1.0 + np.sqrt(1.0 + z64))
    z32 = z64.astype(np.float32)
    s32 = np.floor(np.float32(1.0) + np.sqrt(np.float32(1.0) + z32)).astype(np.float64)
    return s64, s32


def test_fp32_stage_count_differs_only_next_to_an_integer():
    rng = np.random.default_rng(5)
    zmax = ((S_MAX - 1.0) ** 2 - 1.0)  # 1.54 h sigma at the cap
    z = 10.0 ** rng.uniform(-4, np.log10(zmax), 2_000_000)
    s64, s32 = stage_counts(z)
    diff = s64 != s32
    v = 1.0 + np.sqrt(1.0 + z)
    near = np.abs(v - np.round(v)) <= 4 * np.finfo(np.float32).eps * v
    assert (~diff | near).all()  # every disagreement sits next to an integer
    assert (np.abs(s64 - s32) <= 1).all()
    assert diff.mean() < 1e-5
    # and the counts that straddle an integer exactly agree where the value
    # is away from it by more than FP32 rounding
    s = np.arange(2, S_MAX + 1, dtype=np.float64)
    z_int = (s - 1.0) ** 2 - 1.0  # 1 + sqrt(1 + z) == s exactly
    for off in (1e-3, -1e-3):
        zz = z_int * (1.0 + off)
        a, b = stage_counts(zz[zz > 0])
        assert (a == b).all()
