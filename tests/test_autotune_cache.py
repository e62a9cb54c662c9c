"""Host logic of the launch-shape autotuner (no GPU): the JSON cache named by
NYS_TUNE_CACHE is read back, pinned choices are listed and saved, clearing
forgets them, and the on/off switch reports its previous state.  Each case
runs in a fresh interpreter, since the library reads the file once per
process."""

import json
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_02820_gb300 import build
    build.build()


def run(code, env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_cache_file_is_read_pinned_saved_and_cleared(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text('{\n  "rbf_tc16 passes=3 npad=50048 d=16 nvec=128 sms=152": 9,\n'
                    '  "rbf_gemv npad=100096 d=32 nvec=1 sms=152": 1\n}\n')
    got = run("""
        import json
        from paper_2110_02820_gb300 import nyspcg as ny
        first = ny.autotune_choices()
        ny.autotune_set("extra key", 4)
        second = ny.autotune_choices()
        ny.autotune_clear()
        print(json.dumps([first, second, ny.autotune_choices()]))
    """, {"NYS_TUNE_CACHE": str(path)})
    first, second, cleared = got
    assert first == {"rbf_tc16 passes=3 npad=50048 d=16 nvec=128 sms=152": 9,
                     "rbf_gemv npad=100096 d=32 nvec=1 sms=152": 1}
    assert second == dict(first, **{"extra key": 4})
    assert cleared == {}
    # the pinned choice was written back with the others
    assert json.loads(path.read_text()) == second


def test_malformed_cache_stops_at_the_first_bad_entry(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text('{"good": 2, "bad": x, "later": 3}')
    got = run("""
        import json
        from paper_2110_02820_gb300 import nyspcg as ny
        print(json.dumps(ny.autotune_choices()))
    """, {"NYS_TUNE_CACHE": str(path)})
    assert got == {"good": 2}


def test_switch_and_environment_default():
    got = run("""
        import json
        from paper_2110_02820_gb300 import nyspcg as ny
        a = ny.autotune()
        b = ny.autotune(True)
        c = ny.autotune()
        d = ny.pcg_graphs()
        print(json.dumps([a, b, c, d]))
    """, {"NYS_TUNE": "0", "NYS_PCG_GRAPH": "0"})
    assert got == [False, False, True, False]
    got = run("""
        import json
        from paper_2110_02820_gb300 import nyspcg as ny
        print(json.dumps([ny.autotune(), ny.pcg_graphs()]))
    """, {"NYS_TUNE": "", "NYS_PCG_GRAPH": ""})
    assert got == [True, True]


def test_empty_key_is_rejected():
    got = run("""
        import json
        from paper_2110_02820_gb300 import nyspcg as ny
        try:
            ny.autotune_set("", 2)
            print(json.dumps("accepted"))
        except Exception as e:
            print(json.dumps(type(e).__name__))
    """, {})
    assert got != "accepted"
