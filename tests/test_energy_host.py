"""agg_energy_counter against a stand-in NVML (a small C library built here):
device mapping, the counter's value and the error paths. Runs in a child
process because NVML is loaded once per process."""
import os
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_energy_counter_reads_nvml(tmp_path):
    lib = tmp_path / "libfake_nvml.so"
    subprocess.check_call(["gcc", "-shared", "-fPIC", "-O1", "-o", str(lib), os.path.join(ROOT, "tests", "fake_nvml.c")])
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import paper_2606_10030_gb300 as agg
        agg.build()
        assert agg.agg_energy_counter(0) == 1000
        assert agg.agg_energy_counter(0) == 1250
        assert agg.agg_energy_counter(2) == 3000
        for dev, status in ((7, agg.AGG_ERR_CUDA), (9, agg.AGG_ERR_CUDA), (-1, agg.AGG_ERR_INVALID)):
            try:
                agg.agg_energy_counter(dev)
                raise SystemExit("no error for device %%d" %% dev)
            except agg.AggError as e:
                assert e.status == status, (dev, e.status)
        print("ok")
    """ % ROOT)
    env = dict(os.environ, AGG_NVML_LIB=str(lib), CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_missing_nvml_is_an_error(tmp_path):
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import paper_2606_10030_gb300 as agg
        agg.build()
        try:
            agg.agg_energy_counter(0)
        except agg.AggError as e:
            assert e.status == agg.AGG_ERR_CUDA and "NVML" in str(e), str(e)
            print("ok")
    """ % ROOT)
    env = dict(os.environ, AGG_NVML_LIB=str(tmp_path / "no_such_library.so"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
