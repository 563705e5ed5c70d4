"""Buffered scalar queries (GPU): the outputs read one at a time on the host
are the generator's V-stream, across buffer refills, for every variant."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16682_gb300 as m
    from paper_2309_16682_gb300 import build
    build.build()
    m.lib()
    return m


def _plain(vmt, variant, lanes, seed, jump, n, dtype):
    t = vmt.VGenerator(variant, lanes, [seed], [jump]).generate(n, dtype)[0].cpu()
    if t.dtype == torch.uint32:
        return t.view(torch.int32).numpy().view(np.uint32)
    if t.dtype == torch.uint64:
        return t.view(torch.int64).numpy().view(np.uint64)
    return t.numpy()


@pytest.mark.parametrize("variant,dtype", [("mt32", "u32"), ("mt32", "f32"), ("mt64", "u64"), ("mt64", "f64"),
                                           ("sfmt", "u32")])
def test_queries_follow_the_stream(vmt, variant, dtype):
    lanes, seed, jump, n = 4, 31, 12345, 5000
    q = vmt.ScalarGenerator(variant, lanes, seed, jump, dtype, buffer_outputs=1024)
    got = [q.next() for _ in range(700)]                   # single queries
    got = np.concatenate([np.array(got, dtype=q._np), q.take(n - 700 - 300)])
    got = np.concatenate([got, np.array([q.next() for _ in range(300)], dtype=q._np)])
    assert np.array_equal(got, _plain(vmt, variant, lanes, seed, jump, n, dtype))
    q.close()


def test_queries_match_oracle_and_checksum(vmt, oracle_polys):
    q = vmt.ScalarGenerator("mt32", 8, 77, 0, "u32", buffer_outputs=2048)
    got = q.take(9000)
    assert np.array_equal(got, O.vstream(O.MT32, 8, 77, 9000, "u32"))
    # drain: the checksum of the next 5000 single queries
    ref = O.vstream(O.MT32, 8, 77, 14000, "u32")[9000:]
    acc = 0
    for v in ref:
        acc = ((acc ^ int(v)) * 0x100000001B3) & (2**64 - 1)
    assert q.drain(5000) == acc
    q.close()
