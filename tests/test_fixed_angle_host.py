"""Host checks of the FP32 literal-curvature arithmetic (Eq. 10-11): the two float
polynomials for sin(u)/u on the wrapped interval and the fixed-point angle wrap.

The constants are read from the kernel source and the kernel's integer and float steps are
emulated bit for bit in numpy (fused multiply-adds through exact rationals), then compared
with sin(u)/u of the wrapped angle in double: the wrap into [-pi, pi] is Eq. 11's reading
("mod pi" of the half angle), and sin(u)/u is Huber's optimal curvature of 1 - cos."""
import os
import re
from fractions import Fraction

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2005_08661_gb300", "csrc", "k_data.cu")
TURN = 2.0 ** 32 / (2.0 * np.pi)  # fixed-point units per radian


def _src():
    with open(SRC) as f:
        return f.read()


def _radian_coeffs():
    body = _src().split("__device__ __forceinline__ float sinc_wrapped(float u) {")[1].split("}")[0]
    vals = [float(x) for x in re.findall(r"(-?[0-9.]+e?-?[0-9]*)f", body)]
    return vals[::-1]  # c0 .. c5 (Horner starts from c5)


def _turn_coeffs():
    src = _src()
    return [float(re.search(r"constexpr float kSincT%d = (-?[0-9.e-]+)f;" % k, src).group(1)) for k in range(6)]


def f32(x):
    return np.float32(x)


def fma(a, b, c):
    """float fused multiply-add: the exact a*b+c rounded once to float."""
    return np.float32(float(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def horner(c, v):
    p = fma(f32(c[5]), v, f32(c[4]))
    for k in (3, 2, 1, 0):
        p = fma(p, v, f32(c[k]))
    return p


def sinc(u):
    return 1.0 if u == 0.0 else np.sin(u) / u


def wrap(t):
    return t - 2.0 * np.pi * np.rint(t / (2.0 * np.pi))


def to_fixed(ang):
    """the setup's store of a float angle in [-pi, pi]: round-to-nearest, saturating."""
    v = np.rint(float(ang) * (2.0 ** 32 / (2.0 * np.pi)))
    return int(np.clip(v, -2.0 ** 31, 2.0 ** 31 - 1)) & 0xFFFFFFFF


def phase_fixed(w, dtt):
    hi = f32(float(w) * float(dtt))
    lo = fma(w, dtt, -hi)
    return (int(np.rint(float(hi))) + int(np.rint(float(lo)))) & 0xFFFFFFFF


def term_fixed(an, bm, c):
    t = (an - bm) & 0xFFFFFFFF
    bits = ((t >> 9) | (0x7F << 23)) & 0xFFFFFFFF  # funnel shift of {0x7F : t} by 9
    f = np.frombuffer(np.uint32(bits).tobytes(), dtype=np.float32)[0]
    x = f32(f - f32(1.5))
    return horner(c, f32(x * x))


def test_radian_polynomial_matches_wrapped_sinc():
    c = _radian_coeffs()
    assert len(c) == 6
    u = np.linspace(-np.pi - 0.01, np.pi + 0.01, 4001)
    err = max(abs(float(horner(c, f32(f32(x) * f32(x)))) - sinc(float(f32(x)))) for x in u)
    assert err < 3e-7


def test_turn_polynomial_matches_wrapped_sinc():
    c = _turn_coeffs()
    x = np.linspace(-0.5, 0.5, 4001)
    err = max(abs(float(horner(c, f32(f32(t) * f32(t)))) - sinc(2.0 * np.pi * float(f32(t)))) for t in x)
    assert err < 2.5e-7
    # the two fits describe the same function: c_k(turns) = c_k(radians) (2 pi)^(2k) to fit accuracy
    cr = _radian_coeffs()
    assert abs(c[0] - cr[0]) < 1e-7 and abs(c[1] / (cr[1] * (2 * np.pi) ** 2) - 1) < 1e-4


@pytest.mark.parametrize("seed", [0, 1])
def test_fixed_point_wrap_matches_double(seed):
    """sinc(wrap(angle W_dn + w dt - angle W_cm)) through the kernel's fixed-point steps,
    against double, for field values up to +-2 kHz and echo spacings up to 40 ms."""
    rng = np.random.default_rng(seed)
    c = _turn_coeffs()
    worst = 0.0
    for _ in range(3000):
        pn, pm = f32(rng.uniform(-np.pi, np.pi)), f32(rng.uniform(-np.pi, np.pi))
        w = f32(rng.uniform(-2 * np.pi * 2000, 2 * np.pi * 2000))
        dt = float(rng.choice([-2e-3, -8e-3, -10e-3, -40e-3]))
        dtt = f32(dt * TURN)
        an = (to_fixed(pn) + phase_fixed(w, dtt) + 0x80000100) & 0xFFFFFFFF
        got = float(term_fixed(an, to_fixed(pm), c))
        # the same float inputs in double; dt enters as the float dtt the kernel uses
        th = float(pn) + float(w) * float(dtt) / TURN - float(pm)
        worst = max(worst, abs(got - sinc(wrap(th))))
    assert worst < 7e-7


def test_fixed_point_wrap_edges():
    c = _turn_coeffs()
    # a difference of exactly half a turn (either sign) gives sinc(pi) = 0 from both sides
    for pn, pm in [(np.pi, 0.0), (-np.pi, 0.0), (0.0, np.pi), (np.pi, -np.pi)]:
        an = (to_fixed(f32(pn)) + 0x80000100) & 0xFFFFFFFF
        got = float(term_fixed(an, to_fixed(f32(pm)), c))
        assert abs(got - sinc(wrap(float(f32(pn)) - float(f32(pm))))) < 7e-7
    # equal angles: sinc(0) = 1; whole turns of phase vanish
    an = (to_fixed(f32(1.0)) + phase_fixed(f32(1.0), f32(2.0 ** 32)) + 0x80000100) & 0xFFFFFFFF
    assert abs(float(term_fixed(an, to_fixed(f32(1.0)), c)) - 1.0) < 2e-7
    # a plausible mistake -- the half-turn offset left out -- is caught
    an_bad = to_fixed(f32(0.3))
    bad = float(term_fixed(an_bad, to_fixed(f32(0.3)), c))
    assert abs(bad - 1.0) > 0.5


def test_fixed_point_scale_constants_agree():
    """The setup's angle store, the pair table's phase factor and the kernels' conversion
    back to radians all use one turn = 2^32."""
    csrc = os.path.join(os.path.dirname(SRC))
    with open(os.path.join(csrc, "k_setup.cu")) as f:
        setup = f.read()
    with open(os.path.join(csrc, "fm_api.cu")) as f:
        api = f.read()
    store = float(re.search(r"__double2int_rn\(\(double\)ang \* ([0-9.]+)\)", setup).group(1))
    phase = float(re.search(r"pr\.dtt\[pr\.P\] = \(float\)\(pr\.dt\[pr\.P\] \* ([0-9.]+)\)", api).group(1))
    back = float(re.search(r"__float_as_int\(bits\) \* ([0-9.e-]+)f", _src()).group(1))
    assert abs(store / TURN - 1) < 1e-15 and abs(phase / TURN - 1) < 1e-15
    assert abs(back * TURN - 1) < 1e-7
