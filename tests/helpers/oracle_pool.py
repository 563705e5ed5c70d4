"""Oracle work for the wide-sample parity test, run in spawned processes (the
parent has already used the GPU): the first `words` words of the V-stream of
one generator.  The lane polynomials x^(tJ) are computed once per process."""
import oracle as O

_POLYS = {}


def first_words(args):
    variant, M, seed, words = args
    if (variant, M) not in _POLYS:
        J = O.lane_spacing(M)
        _POLYS[(variant, M)] = [O.xpow(variant, t * J) for t in range(1, M)]
    x0 = O.seed_state(variant, seed)
    lanes = [x0] + [O.jump(x0, c) for c in _POLYS[(variant, M)]]
    return O.vstream_words(variant, M, 0, words, lanes=lanes)
