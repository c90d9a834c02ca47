"""Host-side NUMA helpers of the benchmark's page-locked buffers, on fake
sysfs and numa_maps texts (no GPU)."""

import os

from paper_2204_02085_gb300 import hostnuma


def test_cpulists_round_trip():
    assert hostnuma.parse_cpulist("0-3,8,10-11") == {0, 1, 2, 3, 8, 10, 11}
    assert hostnuma.parse_cpulist("") == set() and hostnuma.parse_cpulist(None) == set()
    assert hostnuma.format_cpulist({11, 0, 1, 2, 3, 8, 10}) == "0-3,8,10-11"
    assert hostnuma.format_cpulist(set()) == ""
    assert hostnuma.parse_cpulist(hostnuma.format_cpulist({5})) == {5}


def test_locality_from_sysfs(tmp_path):
    d = tmp_path / "0009:01:00.0"
    d.mkdir()
    (d / "numa_node").write_text("1\n")
    (d / "local_cpulist").write_text("72-143\n")
    loc = hostnuma.locality_of("0009:01:00.0", str(tmp_path))
    assert loc == {"pci": "0009:01:00.0", "node": 1, "local_cpus": "72-143"}
    (d / "numa_node").write_text("-1\n")  # a machine without NUMA
    assert hostnuma.locality_of("0009:01:00.0", str(tmp_path))["node"] is None
    assert hostnuma.locality_of(None, str(tmp_path)) == {"pci": None, "node": None, "local_cpus": None}


def test_cpu_node_from_sysfs(tmp_path):
    c = tmp_path / "cpu7"
    c.mkdir()
    os.symlink(str(tmp_path), str(c / "node1"))
    (c / "online").write_text("1")
    assert hostnuma.cpu_node(7, str(tmp_path)) == 1
    assert hostnuma.cpu_node(8, str(tmp_path)) is None


MAPS = """\
400000 default file=/usr/bin/python3 mapped=100 N0=100 kernelpagesize_kB=64
7f0000000000 default anon=4096 dirty=4096 N0=1024 N1=3072 kernelpagesize_kB=64
7f0100000000 bind:1 anon=16 dirty=16 N1=16 kernelpagesize_kB=64
7f0200000000 default
"""


def test_placement_counts_each_mapping_once():
    maps = hostnuma.parse_numa_maps(MAPS)
    assert [s for s, _ in maps] == [0x400000, 0x7F0000000000, 0x7F0100000000, 0x7F0200000000]
    # two addresses in the second mapping, one in the third
    got = hostnuma.placement([0x7F0000000010, 0x7F0000100000, 0x7F0100000008], numa_maps=MAPS)
    assert got == {0: 1024, 1: 3072 + 16}
    assert hostnuma.placement([0x10], numa_maps=MAPS) == {}  # below every mapping
    assert hostnuma.placement([0x7F0200000000], numa_maps=MAPS) == {}  # no pages yet


def test_current_cpu_is_allowed():
    cpu = hostnuma.current_cpu()
    assert cpu is None or cpu in os.sched_getaffinity(0)
