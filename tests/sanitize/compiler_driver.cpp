// compiler_driver.cpp -- runs the host circuit compiler and frame-program
// builder over a corpus of circuits, for address/undefined-behaviour
// sanitizer builds (tests/test_sanitizers.py). The corpus file holds circuits
// separated by lines "%%"; each is compiled, and valid ones get their frame
// programs built for clusters of 1, 2, 4 and 8 CTAs. Prints one line per
// circuit; exits non-zero only on a sanitizer report (the sanitizers abort).
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    std::ifstream f(argv[1]);
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string all = ss.str();
    std::vector<std::string> circuits;
    size_t pos = 0;
    while (pos <= all.size()) {
        size_t end = all.find("\n%%\n", pos);
        if (end == std::string::npos) end = all.size();
        circuits.push_back(all.substr(pos, end - pos));
        pos = end + 4;
    }
    int ok = 0, rejected = 0;
    for (const std::string &t : circuits) {
        stimgb::HostProgram hp;
        std::string err;
        if (stimgb::compile_circuit(t.data(), t.size(), &hp, &err) != 0) {
            rejected++;
            continue;
        }
        for (int C : {1, 2, 4, 8}) {
            stimgb::FrameProgram fp;
            stimgb::build_frame_program(hp, C, &fp);
        }
        ok++;
    }
    std::printf("compiled %d rejected %d\n", ok, rejected);
    return 0;
}
