"""Host logic of bench.py that needs no GPU: the clock record of the timed region and the
launch-list summary."""
import bench


def test_clock_summary_from_nvml_samples():
    # (SM clock, max clock, NVML clock-event reason bits): sw_power_cap 0x4, hw_slowdown 0x8,
    # sw_thermal_slowdown 0x20, hw_thermal_slowdown 0x40; the idle bit 0x1 is not reported
    c = bench.ClockSampler(0)
    c.source = "nvml"
    c.samples = [(2070.0, 2070.0, 0x0), (2055.0, 2070.0, 0x4 | 0x1), (1980.0, 2070.0, 0x8)]
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["min_sm_mhz"] == 1980.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"] and s["samples"] == 3 and s["source"] == "nvml"


def test_clock_summary_from_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.source = "nvidia-smi"
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"]
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["reasons"] == ["sw_power_cap"] and s["samples"] == 2


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["unsampled"]


def test_launch_summary(tmp_path, capsys):
    # ncu --csv launch list: per kernel launches, total time and share
    p = tmp_path / "launches.csv"
    rows = ['"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
            '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"']
    for i, (name, ns) in enumerate([("k_a", 3000), ("k_b", 1000), ("k_a", 1000)]):
        rows.append('"%d","1","python","h","%s","1","7","(128, 1, 1)","(10, 1, 1)","0","10.3",'
                    '"Command line profiler metrics","gpu__time_duration.sum","ns","%d"' % (i, name, ns))
    p.write_text("\n".join(rows) + "\n")
    bench.summarize_launches(str(p))
    lines = capsys.readouterr().out.splitlines()
    a = next(l for l in lines if l.startswith("k_a"))
    b = next(l for l in lines if l.startswith("k_b"))
    assert a.split()[1:] == ["2", "0.004", "80.00%"] and b.split()[1:] == ["1", "0.001", "20.00%"]
